"""GB300-native dense full-tableau simplex (arXiv 2211.10979, Section III).

The product path is the CUDA library ``libtabsimplex.so`` (C ABI in
``include/tabsimplex.h``); this package binds it with ctypes (``abi``) and adds
a small convenience layer (``solve``, ``Problem``) plus the hook that routes
the library's device allocations through PyTorch's caching allocator.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import abi
from .abi import (LP_ERR_CUDA, LP_ERR_INVALID, LP_ERR_NOMEM, LP_ERR_NUMERIC, LP_ERR_STATE,
                  LP_ERR_TIMEOUT, LP_ITER_LIMIT, LP_LAYOUT_CONDENSED, LP_LAYOUT_FULL, LP_OPTIMAL,
                  LP_PATH_AUTO, LP_PATH_CLUSTER, LP_PATH_HYBRID, LP_PATH_MULTILAUNCH, LP_PATH_TEAM,
                  LP_PATH_PERSISTENT, LP_PREC_FP32, LP_PREC_FP64, LP_RULE_BLAND, LP_RULE_DANTZIG, LP_UNBOUNDED, STATUS_NAMES,
                  lp_create, lp_create_device, lp_destroy, lp_get_pivot_log, lp_get_solution,
                  lp_get_stats, lp_get_tableau, lp_last_error, lp_options, lp_options_init,
                  lp_set_allocator, lp_solve, lp_solve_many, lp_solve_noalloc, lp_stats, lp_version,
                  lp_batch_options, lp_batch_options_init, lp_batch_create, lp_batch_create_device,
                  lp_batch_solve, lp_batch_get, lp_batch_get_tableau, lp_batch_get_stats,
                  lp_batch_destroy, LP_PENDING, lps_options, lps_options_init, lps_open, lps_submit,
                  lps_submit_device, lps_wait, lps_result, lps_release, lps_get_stats, lps_last_error, lps_close,
                  lp_generate_dense)

__all__ = [n for n in dir(abi) if n.startswith(("lp_", "LP_"))] + [
    "STATUS_NAMES", "Solution", "Problem", "solve", "use_torch_allocator", "options",
    "Batch", "BatchSolution", "batch_options", "Server", "ServedResult", "server_options"]

_torch_hooks = None


def use_torch_allocator() -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    if _torch_hooks is not None:
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:   # noqa: BLE001 - reported to the library as NULL
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (abi.ALLOC_FN(_alloc), abi.FREE_FN(_free))
    if abi.lp_set_allocator(hooks[0], hooks[1], None) != 0:
        raise RuntimeError(abi.lp_last_error())
    _torch_hooks = hooks


def options(**kw) -> lp_options:
    """lp_options with the library defaults, then the given fields."""
    o = lp_options_init()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"lp_options has no field {k!r}")
        setattr(o, k, v)
    return o


@dataclass
class Solution:
    status: int
    iters: int
    x: np.ndarray
    y: np.ndarray
    obj: float
    basis: np.ndarray
    stats: dict


class Problem:
    """Owns one lp_t handle (host or device inputs)."""

    def __init__(self, A, b, c, device: bool = False, stream=None):
        if device:
            m, n = A.shape
            self.m, self.n = int(m), int(n)
            self._keep = (A, b, c)          # the library references device inputs
            self.h = lp_create_device(self.m, self.n, A, b, c, stream)
        else:
            A = np.ascontiguousarray(A, dtype=np.float64)
            b = np.ascontiguousarray(b, dtype=np.float64)
            c = np.ascontiguousarray(c, dtype=np.float64)
            self.m, self.n = A.shape
            self.h = lp_create(self.m, self.n, A, b, c)

    def solve(self, opts: lp_options | None = None) -> int:
        st = lp_solve(self.h, opts)
        if st < 0 and st != LP_ERR_TIMEOUT:
            raise RuntimeError(f"lp_solve failed ({STATUS_NAMES.get(st, st)}): {lp_last_error()}")
        return st

    def solution(self) -> Solution:
        x = np.empty(self.n, dtype=np.float64)
        y = np.empty(self.m, dtype=np.float64)
        obj = np.empty(1, dtype=np.float64)
        basis = np.empty(self.m, dtype=np.int32)
        st, it = lp_get_solution(self.h, x, y, obj, basis)
        return Solution(st, it, x, y, float(obj[0]), basis, lp_get_stats(self.h).as_dict())

    def tableau(self) -> np.ndarray:
        T = np.empty((self.m + 1, self.n + self.m + 1), dtype=np.float64)
        st = lp_get_tableau(self.h, T)
        if st != 0:
            raise RuntimeError(lp_last_error())
        return T

    def pivot_log(self, cap: int):
        q = np.empty(cap, dtype=np.int32)
        p = np.empty(cap, dtype=np.int32)
        st, k = lp_get_pivot_log(self.h, q, p, cap)
        if st != 0:
            raise RuntimeError(lp_last_error())
        return q[:k].copy(), p[:k].copy()

    def stats(self) -> dict:
        return lp_get_stats(self.h).as_dict()

    def close(self):
        if getattr(self, "h", None):
            lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_many(problems, opts: lp_options | None = None):
    """Solves several Problems at once (lp_solve_many: a team of blocks per
    LP, one launch); returns the per-LP statuses.  Each Problem then answers
    solution() / tableau() / stats() as after its own solve()."""
    rc, st = lp_solve_many([p.h for p in problems], opts)
    if rc != LP_OPTIMAL:
        raise RuntimeError(f"lp_solve_many failed ({STATUS_NAMES.get(rc, rc)}): {lp_last_error()}")
    return st


def batch_options(**kw) -> lp_batch_options:
    """lp_batch_options with the library defaults, then the given fields."""
    o = lp_batch_options_init()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"lp_batch_options has no field {k!r}")
        setattr(o, k, v)
    return o


@dataclass
class BatchSolution:
    status: np.ndarray
    iters: np.ndarray
    obj: np.ndarray
    x: list          # per LP, views into the packed array
    y: list
    stats: dict


class Batch:
    """Owns one lp_batch_t: many LPs solved together (one block per LP)."""

    def __init__(self, problems=None, *, m=None, n=None, A=None, b=None, c=None, device=False,
                 stream=None):
        if problems is not None:
            m = np.array([p[0].shape[0] for p in problems], dtype=np.int32)
            n = np.array([p[0].shape[1] for p in problems], dtype=np.int32)
            A = np.concatenate([np.ascontiguousarray(p[0], dtype=np.float64).ravel() for p in problems])
            b = np.concatenate([np.asarray(p[1], dtype=np.float64) for p in problems])
            c = np.concatenate([np.asarray(p[2], dtype=np.float64) for p in problems])
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.count = len(self.m)
        self.x_off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.y_off = np.concatenate([[0], np.cumsum(self.m)]).astype(np.int64)
        if device:
            self._keep = (A, b, c)
            self.h = lp_batch_create_device(self.count, self.m, self.n, A, b, c, stream)
        else:
            self._keep = (np.ascontiguousarray(A, dtype=np.float64),
                          np.ascontiguousarray(b, dtype=np.float64),
                          np.ascontiguousarray(c, dtype=np.float64))
            self.h = lp_batch_create(self.count, self.m, self.n, *self._keep)

    def solve(self, opts: lp_batch_options | None = None) -> None:
        st = lp_batch_solve(self.h, opts)
        if st != 0:
            raise RuntimeError(f"lp_batch_solve failed ({STATUS_NAMES.get(st, st)}): {lp_last_error()}")

    def results(self) -> BatchSolution:
        status = np.empty(self.count, dtype=np.int32)
        iters = np.empty(self.count, dtype=np.int64)
        obj = np.empty(self.count, dtype=np.float64)
        x = np.empty(int(self.x_off[-1]), dtype=np.float64)
        y = np.empty(int(self.y_off[-1]), dtype=np.float64)
        if lp_batch_get(self.h, status, iters, obj, x, y) != 0:
            raise RuntimeError(lp_last_error())
        xs = [x[self.x_off[k]:self.x_off[k + 1]] for k in range(self.count)]
        ys = [y[self.y_off[k]:self.y_off[k + 1]] for k in range(self.count)]
        return BatchSolution(status, iters, obj, xs, ys, lp_batch_get_stats(self.h).as_dict())

    def tableau(self, k: int) -> np.ndarray:
        m, n = int(self.m[k]), int(self.n[k])
        T = np.empty((m + 1, n + m + 1), dtype=np.float64)
        if lp_batch_get_tableau(self.h, k, T) != 0:
            raise RuntimeError(lp_last_error())
        return T

    def close(self):
        if getattr(self, "h", None):
            lp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def server_options(**kw) -> lps_options:
    """lps_options with the library defaults, then the given fields."""
    o = lps_options_init()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"lps_options has no field {k!r}")
        setattr(o, k, v)
    return o


@dataclass
class ServedResult:
    status: int
    iters: int
    x: np.ndarray
    y: np.ndarray
    obj: float
    t_submit: float
    t_admit: float
    t_done: float


class Server:
    """Owns one lps_t (request server with continuous batching)."""

    def __init__(self, **opts):
        self.h = lps_open(server_options(**opts))
        self.shapes = {}

    def submit(self, A, b, c) -> int:
        A = np.ascontiguousarray(A, dtype=np.float64)
        m, n = A.shape
        t = lps_submit(self.h, m, n, A, np.ascontiguousarray(b, dtype=np.float64),
                       np.ascontiguousarray(c, dtype=np.float64))
        self.shapes[t] = (m, n)
        return t

    def submit_device(self, m, n, dA, db, dc) -> int:
        t = lps_submit_device(self.h, m, n, dA, db, dc)
        self.shapes[t] = (m, n)
        return t

    def wait(self, ticket, timeout_s=-1.0) -> int:
        return lps_wait(self.h, ticket, timeout_s)

    def result(self, ticket, release=True) -> ServedResult:
        m, n = self.shapes[ticket]
        x = np.empty(n)
        y = np.empty(m)
        obj = np.empty(1)
        times = np.empty(3)
        st, it = lps_result(self.h, ticket, x, y, obj, times)
        if release:
            lps_release(self.h, ticket)
            del self.shapes[ticket]
        return ServedResult(st, it, x, y, float(obj[0]), *times.tolist())

    def stats(self) -> dict:
        return lps_get_stats(self.h).as_dict()

    def last_error(self) -> str:
        return lps_last_error(self.h)

    def close(self):
        if getattr(self, "h", None):
            lps_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve(A, b, c, **opts) -> Solution:
    """Create, solve and read out one LP from host arrays."""
    with Problem(A, b, c) as pr:
        pr.solve(options(**opts))
        return pr.solution()


del ctypes
