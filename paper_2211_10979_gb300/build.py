"""Build the sm_103a shared library in-tree with nvcc (no torch extension).

    python -m paper_2211_10979_gb300.build

produces ``paper_2211_10979_gb300/libtabsimplex.so`` from ``csrc/*.cu`` with
the C ABI of ``include/tabsimplex.h``.  The CUDA runtime is linked statically,
so the library only needs the driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libtabsimplex.so")
SOURCES = ["tabsimplex.cu", "batch.cu", "server.cu", "measure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=default", "-Xcompiler", "-ffp-contract=off", "-shared"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "tabsimplex.h"))
    return out


# Sources of the single-LP pivot kernels' device code (a profile of the
# persistent kernel stays valid while these are unchanged and the launch
# shape recorded with it is the same).
PIVOT_SOURCES = ("tsx_device.cuh", "tsx_kernels.cuh")


def source_digest(names=None) -> str:
    """SHA-256 (first 16 hex digits) over the library's sources and header, or
    over the files with the given base names only."""
    import hashlib
    h = hashlib.sha256()
    for path in sorted(_deps()):
        if names is not None and os.path.basename(path) not in names:
            continue
        if path.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(os.path.basename(path).encode())
            with open(path, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, defines=(), out: str | None = None) -> str:
    """Compile the library (skipped when up to date).  `defines` are extra -D
    flags for tuning builds (e.g. "TSX_ROWS_IN_FLIGHT=4"); `out` another path."""
    target = out or LIB
    if not force and not defines and out is None and up_to_date():
        return LIB
    tag = f"{os.getpid()}"
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    compile_flags = [f for f in FLAGS if f != "-shared"]
    procs, objs = [], []
    for src in SOURCES:   # translation units compiled in parallel
        obj = os.path.join(objdir, f"{os.path.splitext(src)[0]}.{tag}.o")
        cmd = [nvcc(), *ARCH, *compile_flags, *[f"-D{d}" for d in defines], "-I", INCLUDE, "-I", CSRC,
               "-c", "-o", obj, os.path.join(CSRC, src)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    try:
        codes = [p.wait() for p in procs]
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc")
        tmp = target + f".tmp{tag}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs], check=True)
        os.replace(tmp, target)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return target


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
