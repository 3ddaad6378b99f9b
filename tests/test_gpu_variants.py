"""Compile-time variants of the pivot kernel vs the CPU oracle (needs a GPU).

The default build streams the rank-1 update through registers (16 rows in
flight per warp).  `TSX_TMA=1` builds the alternative update of the condensed
tableau: every warp copies its slots' rows into a ring of shared-memory stages
with `cp.async.bulk` and one mbarrier per stage, and runs the fused
multiply-adds from shared memory.  The variant is built into its own library
file and the whole FP64 parity module (pivot sequence, basis and tableau equal
to the oracle's) runs against it in a child process, so that this process
keeps the default library.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

VARIANTS = {
    # one block of 256 threads per SM: 8 rows x 3 stages (24 KB) per warp
    "bulk_copy_ring": ("TSX_TMA=1", "TSX_TMA_ROWS=8", "TSX_TMA_STAGES=3"),
    # two blocks per SM: 4 rows x 3 stages (12 KB) per warp, 128 registers
    "bulk_copy_ring_2_blocks": ("TSX_TMA=1", "TSX_SM_THREADS=512", "TSX_TMA_ROWS=4", "TSX_TMA_STAGES=3"),
}


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_variant_parity(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10979_gb300 import build
    out = os.path.join(build.PKG, "_build", f"libtabsimplex_{name}.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    build.build(defines=VARIANTS[name], out=out)
    code = textwrap.dedent(f"""
        import sys
        sys.path[:0] = [{ROOT!r}, {os.path.join(ROOT, 'tests')!r}]
        from paper_2211_10979_gb300 import abi
        abi.load({out!r})          # every later load() returns this library
        import pytest
        sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "gpu",
                              {os.path.join(ROOT, 'tests', 'test_gpu_parity.py')!r}]))
    """)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert " passed" in r.stdout
