"""ctypes binding of the C ABI in include/tabsimplex.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: the whole solve runs in the library's CUDA kernels.
Loading fails loudly when the shared library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtabsimplex.so")

LP_OPTIMAL, LP_UNBOUNDED, LP_ITER_LIMIT, LP_ERR_NUMERIC = 0, 1, 2, 3
LP_ERR_INVALID, LP_ERR_NOMEM, LP_ERR_CUDA, LP_ERR_TIMEOUT, LP_ERR_STATE = -1, -2, -3, -4, -5
STATUS_NAMES = {0: "OPTIMAL", 1: "UNBOUNDED", 2: "ITER_LIMIT", 3: "NUMERIC", -1: "INVALID",
                -2: "NOMEM", -3: "CUDA", -4: "TIMEOUT", -5: "STATE", 100: "PENDING"}
LP_RULE_DANTZIG, LP_RULE_BLAND = 0, 1
LP_LAYOUT_CONDENSED, LP_LAYOUT_FULL = 0, 1
LP_PATH_AUTO, LP_PATH_PERSISTENT, LP_PATH_MULTILAUNCH, LP_PATH_TEAM, LP_PATH_CLUSTER, LP_PATH_HYBRID = 0, 1, 2, 3, 4, 5
LP_PREC_FP64, LP_PREC_FP32 = 0, 1

# every symbol include/tabsimplex.h declares
EXPORTS = ("lp_options_init", "lp_create", "lp_create_device", "lp_solve", "lp_get_solution",
           "lp_get_tableau", "lp_get_pivot_log", "lp_get_stats", "lp_destroy", "lp_last_error",
           "lp_set_allocator", "lp_version", "lp_solve_noalloc", "lp_solve_many", "lp_batch_options_init",
           "lp_batch_create", "lp_batch_create_device", "lp_batch_solve", "lp_batch_get",
           "lp_batch_get_tableau", "lp_batch_get_stats", "lp_batch_destroy", "lps_options_init",
           "lps_open", "lps_submit", "lps_submit_device", "lps_wait", "lps_result", "lps_release",
           "lps_get_stats", "lps_last_error", "lps_close", "lp_generate_dense",
           "lp_measure_fp64_fma_rate", "lp_measure_fp64_op_rate")
LP_PENDING = 100

# capacity of the library's fixed work-buffer array used by lp_solve_noalloc
LP_NOALLOC_SCRATCH_BYTES = 2 * 1024 * 1024


class lp_options(ctypes.Structure):
    _fields_ = [
        ("rule", ctypes.c_int),
        ("eps_d", ctypes.c_double),
        ("eps_p", ctypes.c_double),
        ("max_iters", ctypes.c_longlong),
        ("k_cyc", ctypes.c_int),
        ("barrier_timeout_ns", ctypes.c_longlong),
        ("path", ctypes.c_int),
        ("skip_zero_columns", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("blocks", ctypes.c_int),
        ("log_capacity", ctypes.c_longlong),
        ("stream", ctypes.c_void_p),
        ("precision", ctypes.c_int),
        ("eps_d_fp32", ctypes.c_double),
        ("eps_p_fp32", ctypes.c_double),
        ("recover_tol", ctypes.c_double),
        ("cleanup_max", ctypes.c_int),
        ("layout", ctypes.c_int),
        ("gpu_share", ctypes.c_double),
        ("cpu_threads", ctypes.c_int),
    ]


class lp_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_longlong),
        ("build_ms", ctypes.c_double),
        ("pivot_ms", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
        ("dense_update_bytes", ctypes.c_double),
        ("update_bytes", ctypes.c_double),
        ("path", ctypes.c_int),
        ("grid", ctypes.c_int),
        ("block", ctypes.c_int),
        ("ld", ctypes.c_int),
        ("phase_ms", ctypes.c_double * 6),
        ("precision", ctypes.c_int),
        ("pivot_status", ctypes.c_int),
        ("k", ctypes.c_int),
        ("cleanup_pivots", ctypes.c_int),
        ("recover_ms", ctypes.c_double),
        ("primal_violation", ctypes.c_double),
        ("dual_violation", ctypes.c_double),
        ("gap", ctypes.c_double),
        ("layout", ctypes.c_int),
        ("create_copy_ms", ctypes.c_double),
        ("create_check_ms", ctypes.c_double),
        ("create_wall_ms", ctypes.c_double),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(self.phase_ms)
        return d


class lp_batch_options(ctypes.Structure):
    _fields_ = [
        ("threads", ctypes.c_int),
        ("rule", ctypes.c_int),
        ("eps_d", ctypes.c_double),
        ("eps_p", ctypes.c_double),
        ("max_iters", ctypes.c_longlong),
        ("k_cyc", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("keep_tableaux", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class lp_batch_stats(ctypes.Structure):
    _fields_ = [
        ("solve_ms", ctypes.c_double),
        ("total_pivots", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("buckets", ctypes.c_int),
        ("threads", ctypes.c_int * 5),
        ("lps_per_class", ctypes.c_int * 5),
        ("tune_ms", ctypes.c_double),
        ("graph", ctypes.c_int),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["threads"] = list(self.threads)
        d["lps_per_class"] = list(self.lps_per_class)
        return d


class lps_options(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_longlong),
        ("workers", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("batch_small", ctypes.c_int),
        ("batch_max", ctypes.c_int),
        ("small_max_dim", ctypes.c_int),
        ("blocks_per_lp", ctypes.c_int),
        ("batch_max_bytes", ctypes.c_longlong),
        ("path", ctypes.c_int),
        ("team_blocks", ctypes.c_int),
        ("continuous", ctypes.c_int),
    ]


class lps_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong),
        ("completed", ctypes.c_longlong),
        ("wall_s", ctypes.c_double),
        ("lat_p50_ms", ctypes.c_double),
        ("lat_p99_ms", ctypes.c_double),
        ("lat_mean_ms", ctypes.c_double),
        ("lat_max_ms", ctypes.c_double),
        ("queue_p50_ms", ctypes.c_double),
        ("queue_p99_ms", ctypes.c_double),
        ("batches", ctypes.c_longlong),
        ("batched_lps", ctypes.c_longlong),
        ("peak_bytes", ctypes.c_longlong),
        ("waves", ctypes.c_longlong),
        ("wave_lps", ctypes.c_longlong),
        ("wave_ms", ctypes.c_double),
        ("wave_kernel_ms", ctypes.c_double),
        ("wave_create_ms", ctypes.c_double),
        ("wave_wait_ms", ctypes.c_double),
        ("wave_launch_ms", ctypes.c_double),
        ("wait_p50_ms", ctypes.c_double),
        ("wait_p99_ms", ctypes.c_double),
        ("run_p50_ms", ctypes.c_double),
        ("run_p99_ms", ctypes.c_double),
        ("post_p50_ms", ctypes.c_double),
        ("post_p99_ms", ctypes.c_double),
        ("lane_lps", ctypes.c_longlong),
        ("lane_launches", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the shared library (raises if it is missing: build it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_2211_10979_gb300.build` "
                "(the solver has no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        llp = ctypes.POINTER(ctypes.c_longlong)
        sig = {
            "lp_options_init": (None, [ctypes.POINTER(lp_options)]),
            "lp_create": (vp, [ctypes.c_int, ctypes.c_int, vp, vp, vp]),
            "lp_create_device": (vp, [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]),
            "lp_solve": (ctypes.c_int, [vp, ctypes.POINTER(lp_options)]),
            "lp_solve_many": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(lp_options),
                                             ctypes.POINTER(ctypes.c_int)]),
            "lp_get_solution": (ctypes.c_int, [vp, vp, vp, vp, vp, llp]),
            "lp_get_tableau": (ctypes.c_int, [vp, vp]),
            "lp_get_pivot_log": (ctypes.c_int, [vp, vp, vp, ctypes.c_longlong, llp]),
            "lp_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(lp_stats)]),
            "lp_destroy": (None, [vp]),
            "lp_last_error": (ctypes.c_char_p, []),
            "lp_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, vp]),
            "lp_version": (ctypes.c_char_p, []),
            "lp_solve_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                                ctypes.c_longlong, vp, ctypes.POINTER(lp_options),
                                                llp]),
            "lp_batch_options_init": (None, [ctypes.POINTER(lp_batch_options)]),
            "lp_batch_create": (vp, [ctypes.c_int, vp, vp, vp, vp, vp]),
            "lp_batch_create_device": (vp, [ctypes.c_int, vp, vp, vp, vp, vp, vp]),
            "lp_batch_solve": (ctypes.c_int, [vp, ctypes.POINTER(lp_batch_options)]),
            "lp_batch_get": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "lp_batch_get_tableau": (ctypes.c_int, [vp, ctypes.c_int, vp]),
            "lp_batch_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(lp_batch_stats)]),
            "lp_batch_destroy": (None, [vp]),
            "lps_options_init": (None, [ctypes.POINTER(lps_options)]),
            "lps_open": (vp, [ctypes.POINTER(lps_options)]),
            "lps_submit": (ctypes.c_longlong, [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]),
            "lps_submit_device": (ctypes.c_longlong, [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]),
            "lps_wait": (ctypes.c_int, [vp, ctypes.c_longlong, ctypes.c_double]),
            "lps_result": (ctypes.c_int, [vp, ctypes.c_longlong, vp, vp, vp, llp, vp]),
            "lps_release": (ctypes.c_int, [vp, ctypes.c_longlong]),
            "lps_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(lps_stats)]),
            "lps_last_error": (ctypes.c_char_p, [vp]),
            "lps_close": (None, [vp]),
            "lp_generate_dense": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, vp, vp, vp, vp]),
            "lp_measure_fp64_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, vp,
                                                        ctypes.POINTER(ctypes.c_double),
                                                        ctypes.POINTER(ctypes.c_double)]),
            "lp_measure_fp64_op_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_longlong, vp, ctypes.POINTER(ctypes.c_double),
                                                       ctypes.POINTER(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        del dp, ip
        _lib = lib
        return lib


def _ptr(a):
    """Address of a numpy array, a torch tensor, an int address, or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


# ------------------------------------------------------------- entry points
def lp_options_init() -> lp_options:
    o = lp_options()
    load().lp_options_init(ctypes.byref(o))
    return o


def lp_last_error() -> str:
    return (load().lp_last_error() or b"").decode()


def lp_version() -> str:
    return load().lp_version().decode()


def lp_create(m: int, n: int, A, b, c) -> int:
    """A, b, c: C-contiguous float64 host arrays. Returns the handle (int)."""
    h = load().lp_create(int(m), int(n), _ptr(A), _ptr(b), _ptr(c))
    if not h:
        raise ValueError(lp_last_error())
    return h


def lp_create_device(m: int, n: int, dA, db, dc, stream=None) -> int:
    """dA, db, dc: device float64 buffers (torch tensors or addresses)."""
    h = load().lp_create_device(int(m), int(n), _ptr(dA), _ptr(db), _ptr(dc), stream)
    if not h:
        raise ValueError(lp_last_error())
    return h


def lp_solve(h: int, opts: lp_options | None = None) -> int:
    return int(load().lp_solve(h, ctypes.byref(opts) if opts is not None else None))


def lp_solve_many(handles, opts: lp_options | None = None):
    """Solves the LPs of the given handles at once; returns (call status,
    list of per-LP statuses)."""
    n = len(handles)
    arr = (ctypes.c_void_p * max(1, n))(*handles)
    st = (ctypes.c_int * max(1, n))()
    rc = load().lp_solve_many(arr, n, ctypes.byref(opts) if opts is not None else None, st)
    return int(rc), [int(st[k]) for k in range(n)]


def lp_get_solution(h: int, x=None, y=None, obj=None, basis=None):
    """Fills the given host arrays (numpy); returns (status, iters)."""
    it = ctypes.c_longlong(0)
    st = load().lp_get_solution(h, _ptr(x), _ptr(y), _ptr(obj), _ptr(basis), ctypes.byref(it))
    return int(st), int(it.value)


def lp_get_tableau(h: int, T) -> int:
    return int(load().lp_get_tableau(h, _ptr(T)))


def lp_get_pivot_log(h: int, q, p, cap: int):
    cnt = ctypes.c_longlong(0)
    st = load().lp_get_pivot_log(h, _ptr(q), _ptr(p), int(cap), ctypes.byref(cnt))
    return int(st), int(cnt.value)


def lp_get_stats(h: int) -> lp_stats:
    s = lp_stats()
    st = load().lp_get_stats(h, ctypes.byref(s))
    if st != 0:
        raise RuntimeError(lp_last_error())
    return s


def lp_destroy(h: int) -> None:
    if h:
        load().lp_destroy(h)


def lp_solve_noalloc(m: int, n: int, dA, db, dc, dT, ld: int, dbasis,
                     opts: lp_options | None = None):
    """Solve into caller-owned device buffers without any device allocation.

    dA, db, dc: device inputs; dT: device (m+1) x ld float64 output; dbasis:
    device int32 output (m).  Returns (status, iters).  The C function cannot
    see buffer sizes, so torch tensors are checked here first (CUDA, dtype,
    contiguous, large enough) and a mismatch raises ValueError before any
    device work; plain integer addresses are passed through unchecked."""
    need = (("dA", dA, "float64", int(m) * int(n)), ("db", db, "float64", int(m)),
            ("dc", dc, "float64", int(n)), ("dT", dT, "float64", (int(m) + 1) * int(ld)),
            ("dbasis", dbasis, "int32", int(m)))
    for name, t, dtype, count in need:
        if t is None or isinstance(t, int) or not hasattr(t, "is_cuda"):
            if t is not None and not isinstance(t, int):
                raise ValueError(f"lp_solve_noalloc: {name} must be a CUDA tensor or a device address")
            continue
        if not t.is_cuda:
            raise ValueError(f"lp_solve_noalloc: {name} is not on a CUDA device")
        if str(t.dtype) != f"torch.{dtype}":
            raise ValueError(f"lp_solve_noalloc: {name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"lp_solve_noalloc: {name} must be contiguous")
        if t.numel() < count:
            raise ValueError(f"lp_solve_noalloc: {name} holds {t.numel()} elements, needs {count}")
    it = ctypes.c_longlong(0)
    st = load().lp_solve_noalloc(int(m), int(n), _ptr(dA), _ptr(db), _ptr(dc), _ptr(dT), int(ld),
                                 _ptr(dbasis), ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(it))
    return int(st), int(it.value)


def lp_set_allocator(alloc_fn, free_fn, ctx=None) -> int:
    return int(load().lp_set_allocator(alloc_fn, free_fn, ctx))


# ------------------------------------------------------------- batched solve
def lp_batch_options_init() -> lp_batch_options:
    o = lp_batch_options()
    load().lp_batch_options_init(ctypes.byref(o))
    return o


def lp_batch_create(count: int, m, n, A, b, c) -> int:
    """m, n: int32 host arrays; A, b, c: packed float64 host arrays."""
    h = load().lp_batch_create(int(count), _ptr(m), _ptr(n), _ptr(A), _ptr(b), _ptr(c))
    if not h:
        raise ValueError(lp_last_error())
    return h


def lp_batch_create_device(count: int, m, n, dA, db, dc, stream=None) -> int:
    h = load().lp_batch_create_device(int(count), _ptr(m), _ptr(n), _ptr(dA), _ptr(db), _ptr(dc), stream)
    if not h:
        raise ValueError(lp_last_error())
    return h


def lp_batch_solve(h: int, opts: lp_batch_options | None = None) -> int:
    return int(load().lp_batch_solve(h, ctypes.byref(opts) if opts is not None else None))


def lp_batch_get(h: int, status=None, iters=None, obj=None, x=None, y=None) -> int:
    return int(load().lp_batch_get(h, _ptr(status), _ptr(iters), _ptr(obj), _ptr(x), _ptr(y)))


def lp_batch_get_tableau(h: int, index: int, T) -> int:
    return int(load().lp_batch_get_tableau(h, int(index), _ptr(T)))


def lp_batch_get_stats(h: int) -> lp_batch_stats:
    s = lp_batch_stats()
    if load().lp_batch_get_stats(h, ctypes.byref(s)) != 0:
        raise RuntimeError(lp_last_error())
    return s


def lp_batch_destroy(h: int) -> None:
    if h:
        load().lp_batch_destroy(h)


# ------------------------------------------------------------- request server
def lps_options_init() -> lps_options:
    o = lps_options()
    load().lps_options_init(ctypes.byref(o))
    return o


def lps_open(opts: lps_options | None = None) -> int:
    h = load().lps_open(ctypes.byref(opts) if opts is not None else None)
    if not h:
        raise RuntimeError(lp_last_error())
    return h


def lps_submit(sv: int, m: int, n: int, A, b, c) -> int:
    t = load().lps_submit(sv, int(m), int(n), _ptr(A), _ptr(b), _ptr(c))
    if t < 0:
        raise ValueError(lp_last_error())
    return int(t)


def lps_submit_device(sv: int, m: int, n: int, dA, db, dc) -> int:
    t = load().lps_submit_device(sv, int(m), int(n), _ptr(dA), _ptr(db), _ptr(dc))
    if t < 0:
        raise ValueError(lp_last_error())
    return int(t)


def lps_wait(sv: int, ticket: int, timeout_s: float = -1.0) -> int:
    return int(load().lps_wait(sv, int(ticket), float(timeout_s)))


def lps_result(sv: int, ticket: int, x=None, y=None, obj=None, times=None):
    it = ctypes.c_longlong(0)
    st = load().lps_result(sv, int(ticket), _ptr(x), _ptr(y), _ptr(obj), ctypes.byref(it), _ptr(times))
    return int(st), int(it.value)


def lps_release(sv: int, ticket: int) -> int:
    return int(load().lps_release(sv, int(ticket)))


def lps_get_stats(sv: int) -> lps_stats:
    s = lps_stats()
    if load().lps_get_stats(sv, ctypes.byref(s)) != 0:
        raise RuntimeError(lp_last_error())
    return s


def lps_last_error(sv: int) -> str:
    msg = load().lps_last_error(sv)
    return msg.decode() if msg else ""


def lps_close(sv: int) -> None:
    if sv:
        load().lps_close(sv)


def lp_measure_fp64_fma_rate(blocks: int, threads: int, iters: int, stream=None):
    """Measurement helper: (launch ms, FP64 fma per second) of a DFMA-chain
    kernel on the current device."""
    ms, rate = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().lp_measure_fp64_fma_rate(int(blocks), int(threads), int(iters), stream,
                                         ctypes.byref(ms), ctypes.byref(rate))
    if st != 0:
        raise RuntimeError(lp_last_error())
    return ms.value, rate.value


def lp_measure_fp64_op_rate(op: int, lanes: int, blocks: int, threads: int, iters: int, stream=None):
    """Measurement helper: (launch ms, warp instructions per second) of fma
    (op 0) or division (op 1) chains with `lanes` active lanes per warp."""
    ms, rate = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().lp_measure_fp64_op_rate(int(op), int(lanes), int(blocks), int(threads), int(iters), stream,
                                        ctypes.byref(ms), ctypes.byref(rate))
    if st != 0:
        raise RuntimeError(lp_last_error())
    return ms.value, rate.value


def lp_generate_dense(m: int, n: int, seed: int, dA, db, dc, stream=None) -> int:
    return int(load().lp_generate_dense(int(m), int(n), int(seed), _ptr(dA), _ptr(db), _ptr(dc), stream))
