"""The C-ABI library loads and exports what include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lp\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2211_10979_gb300 import build
    build.build()
    from paper_2211_10979_gb300 import abi
    return abi.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2211_10979_gb300 import abi
    declared = _declared_functions()
    assert declared == set(abi.EXPORTS), declared ^ set(abi.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_options_defaults_roundtrip(lib):
    import paper_2211_10979_gb300 as tsx
    o = tsx.lp_options_init()
    assert o.rule == 0 and o.eps_d == 1e-9 and o.eps_p == 1e-9 and o.max_iters == -1
    assert o.k_cyc == 50 and o.barrier_timeout_ns == 2_000_000_000 and o.path == 0
    assert o.skip_zero_columns == 1 and o.threads == 0 and o.blocks == 0
    assert o.log_capacity == 0 and o.stream is None
    assert o.precision == tsx.LP_PREC_FP64 and o.eps_d_fp32 == 1e-5 and o.eps_p_fp32 == 1e-6
    assert o.recover_tol == 1e-9 and o.cleanup_max == 1000
    assert o.gpu_share == 0.95 and o.cpu_threads == 0
    assert "sm_103a" in tsx.lp_version()


def test_host_side_validation_without_gpu(lib):
    import paper_2211_10979_gb300 as tsx
    A = np.ones((2, 2))
    b = np.ones(2)
    for m, n in ((0, 2), (2, 0), (-1, 3)):
        with pytest.raises(ValueError, match="m > 0 and n > 0"):
            tsx.lp_create(m, n, A, b, b)
    with pytest.raises(ValueError, match="NULL"):
        tsx.lp_create(2, 2, None, b, b)
    assert tsx.lp_solve(0) == tsx.LP_ERR_INVALID
    assert tsx.lp_get_solution(0) == (tsx.LP_ERR_INVALID, 0)
    tsx.lp_destroy(0)
    # allocator hooks come in pairs
    from paper_2211_10979_gb300 import abi
    assert lib.lp_set_allocator(abi.ALLOC_FN(lambda *a: None), abi.FREE_FN(0), None) == -1
    assert "both" in tsx.lp_last_error()
    assert lib.lp_set_allocator(abi.ALLOC_FN(0), abi.FREE_FN(0), None) == 0


def test_missing_library_fails_loudly(tmp_path):
    from paper_2211_10979_gb300 import abi
    saved = abi._lib
    abi._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            abi.load(str(tmp_path / "nope.so"))
    finally:
        abi._lib = saved
