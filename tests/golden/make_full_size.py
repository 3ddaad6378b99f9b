"""Write the full-size oracle goldens (whole solves at the benchmark's sizes).

Every stored value comes from the CPU oracle (``oracle/``) run to completion on
the seeded generator's LP (``lpgen.dense_lp``); nothing here touches the GPU
library.  Run from the repository root:

    python tests/golden/make_full_size.py            # all cases, in parallel
    python tests/golden/make_full_size.py 8192x8192s1

Each case writes ``tests/golden/full_size/<m>x<n>_seed<k>.json`` with
  - the oracle's status, pivot count and objective (Section III,
    Iterate/Finalization Step), the objective as a hex float;
  - the whole (q, p) pivot log (Steps 1 and 2 of every pivot);
  - the final basis, as the rows whose basic variable is no longer their
    slack (row i of 0..m-1 -> variable index; every other row keeps its
    slack n + i);
  - x and y as their nonzero entries, [index, hex float];
  - a SHA-256 of the LP's bytes (lpgen.lp_digest);
  - the instance's separation record: for every pivot the oracle also reports
    the gap between the chosen objective-row entry and the next candidate,
    and between the minimum ratio and the next eligible ratio.  The instance
    counts as non-degenerate when, at every pivot, both gaps exceed
    1e-9 * max(1, |chosen value|), no minimum ratio is <= 0, and no pivot ran
    under Bland's rule; exact parity of the pivot sequence is then expected
    of any correct implementation, whatever the order of its comparisons.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "full_size")
GAP_REL = 1e-9

# (m, n, seed, what the case serves, generator: lpgen.dense_lp or lpgen.diag_dominant_lp)
CASES = {
    "8192x8192s1": (8192, 8192, 1, "bench size, FP64 parity", "dense_lp"),
    "8192x8192s2": (8192, 8192, 2, "bench size, FP64 parity", "dense_lp"),
    "8192x8192s3": (8192, 8192, 3, "bench size, FP64 parity", "dense_lp"),
    "4096x16384s1": (4096, 16384, 1, "aspect-ratio bench size, FP64 parity", "dense_lp"),
    "16384x16384s1": (16384, 16384, 1, "precision config: FP64 reference objective", "dense_lp"),
    "diag2048s1": (2048, 2048, 1, "FP64 recovery of a basis with k = 2048 structurals", "diag_dominant_lp"),
    "diag4096s1": (4096, 4096, 1, "FP64 recovery of a basis with k = 4096 structurals", "diag_dominant_lp"),
}


def path_of(m: int, n: int, seed: int, gen: str = "dense_lp") -> str:
    prefix = "" if gen == "dense_lp" else "diag_"
    return os.path.join(OUT, f"{prefix}{m}x{n}_seed{seed}.json")


def _rel_gap_summary(gap: np.ndarray, base: np.ndarray):
    """Smallest gap / max(1, |base|) and the pivot where it occurs."""
    rel = gap / np.maximum(1.0, np.abs(base))
    rel = np.where(np.isnan(rel), np.inf, rel)
    if rel.size == 0:
        return None, None
    k = int(np.argmin(rel))
    v = float(rel[k])
    return (v if np.isfinite(v) else None), k


def run_case(name: str) -> str:
    import lpgen
    import oracle

    m, n, seed, what, gen = CASES[name]
    A, b, c = getattr(lpgen, gen)(m, n, seed)
    t0 = time.time()
    res, tr = oracle.solve_traced(A, b, c)
    secs = time.time() - t0
    k = res.iters
    dmin, dk = _rel_gap_summary(tr.dgap, tr.dval)
    rmin, rk = _rel_gap_summary(tr.rgap, tr.theta)
    nonpos = int(np.sum(tr.theta <= 0.0))
    bland = int(np.sum(np.isnan(tr.dgap)))
    non_degenerate = (bland == 0 and nonpos == 0
                      and (dmin is None or dmin > GAP_REL)
                      and (rmin is None or rmin > GAP_REL))
    basis = res.basis.astype(np.int64)
    slack = n + np.arange(m)
    moved = np.nonzero(basis != slack)[0]
    xnz = np.nonzero(res.x)[0]
    ynz = np.nonzero(res.y)[0]
    rec = {
        "what": what,
        "generator": f"lpgen.{gen}(m, n, seed)",
        "m": m, "n": n, "seed": seed,
        "lp_sha256": lpgen.lp_digest(A, b, c),
        "oracle": "oracle.solve_traced, default options (Dantzig, eps 1e-9, k_cyc 50)",
        "status": oracle.STATUS_NAMES[res.status],
        "iters": k,
        "obj": float(res.obj).hex(),
        "obj_decimal": repr(float(res.obj)),
        "qlog": res.qlog.tolist(),
        "plog": res.plog.tolist(),
        "basis_moved": [[int(i), int(basis[i])] for i in moved],
        "x_nonzero": [[int(j), float(res.x[j]).hex()] for j in xnz],
        "y_nonzero": [[int(i), float(res.y[i]).hex()] for i in ynz],
        "separation": {
            "rule": "both gaps > 1e-9 * max(1, |chosen value|) at every pivot, "
                    "no minimum ratio <= 0, no pivot under Bland's rule",
            "min_objective_gap_rel": dmin, "objective_at_pivot": dk,
            "min_ratio_gap_rel": rmin, "ratio_at_pivot": rk,
            "min_ratio": float(np.min(tr.theta)) if k else None,
            "nonpositive_ratio_pivots": nonpos,
            "bland_pivots": bland,
            "non_degenerate": bool(non_degenerate),
        },
        "oracle_seconds": round(secs, 1),
    }
    os.makedirs(OUT, exist_ok=True)
    p = path_of(m, n, seed, gen)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(rec, f, separators=(",", ":"))
        f.write("\n")
    os.replace(tmp, p)
    return f"{name}: {rec['status']} {k} pivots, obj {res.obj!r}, {secs:.0f} s, " \
           f"non-degenerate {non_degenerate}"


def main(argv):
    names = argv or list(CASES)
    for nm in names:
        if nm not in CASES:
            raise SystemExit(f"unknown case {nm}; known: {', '.join(CASES)}")
    if len(names) == 1:
        print(run_case(names[0]), flush=True)
        return
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for line in pool.imap_unordered(run_case, names):
            print(line, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
