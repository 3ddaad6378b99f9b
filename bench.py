#!/usr/bin/env python3
"""Benchmark: pivots/s of the dense full-tableau simplex on GB300.

One step = one whole solve of a seeded dense LP (default m = n = 8192, FP64,
A_ij ~ U[1,10), b_i ~ U[100,1000), c_j ~ U[1,10)): tableau build (Section III
Initialization Step), every pivot (Steps 1-3) until optimal, and the solution
read-out, through the library's C ABI.  The inputs (A, b, c) are resident in
HBM before the timed region (``value``); ``e2e`` repeats the solve from pinned
HOST buffers with the host<->device copies inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--m 8192 --n 8192]
    python bench.py --impl reference ...   # the CPU oracle arm

Multi-GPU (torchrun, one process per GPU): every rank solves its own seeds
(independent LPs, no data-path collective); value = total pivots of all ranks
divided by the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lpgen  # noqa: E402

METRIC = "pivots/s"
UNIT = "pivots/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--m", type=int, default=8192)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--seeds", type=int, default=3, help="distinct LPs cycled through the steps")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--skip-zero", type=int, default=1)
    ap.add_argument("--path", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ ranks
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seeds(rank: int, nseeds: int):
    """Seeds of a rank: rank r solves seeds r*nseeds+1 .. r*nseeds+nseeds."""
    return [rank * nseeds + k + 1 for k in range(nseeds)]


def combine_ranks(per_rank):
    """per_rank: list of (pivots, seconds).  Whole-job throughput = total pivots
    over the slowest rank's time (max over ranks)."""
    total = sum(p for p, _ in per_rank)
    tmax = max(t for _, t in per_rank)
    return total / tmax, tmax


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profile_traffic(m, n):
    """ncu DRAM bytes per pivot of the update kernel, if a summary for this
    exact kernel build and workload is committed under profiles/."""
    path = os.path.join(ROOT, "profiles", "traffic_k_pivot_persistent.txt")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    key = f"{m}x{n}"
    ent = d.get(key)
    if not ent:
        return None
    from paper_2211_10979_gb300 import build as b
    if ent.get("source_digest") != b.source_digest():
        return None   # the kernel changed since the counters were taken
    return ent


def oracle_sample(m, n, seed, budget_s):
    """The CPU oracle on a bounded sample of the workload: the tableau build and
    the first K pivots of the same LP, K chosen so the pivots take ~budget_s."""
    import oracle
    A, b, c = lpgen.dense_lp(m, n, seed)
    t0 = time.perf_counter()
    T, basis = oracle.build_tableau(A, b, c)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    st, it, _, _ = oracle.solve_tableau(T, basis, m, n, oracle.Options(max_iters=1), log_cap=1)
    t1 = time.perf_counter() - t0
    k_more = max(1, int(budget_s / max(t1, 1e-6)) - 1)
    t0 = time.perf_counter()
    st, it2, _, _ = oracle.solve_tableau(T, basis, m, n, oracle.Options(max_iters=k_more), log_cap=1)
    t2 = time.perf_counter() - t0
    pivots = it + it2
    secs = t1 + t2
    return {"value": pivots / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {pivots} pivots of the {m}x{n} seed-{seed} LP "
                      f"(single-threaded C, FP64; tableau build {t_build:.2f}s untimed)",
            "seconds": secs, "pivots": pivots}


# ---------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    budget = max(2.0, args.cpu_seconds / 3.0)
    for _ in range(args.warmup):
        oracle_sample(args.m, args.n, 1, 0.5)
    vals, secs, pivs = [], 0.0, 0
    for k in range(args.steps):
        r = oracle_sample(args.m, args.n, 1 + k % args.seeds, budget)
        vals.append(r["value"])
        secs += r["seconds"]
        pivs += r["pivots"]
    value = pivs / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"dense LP m={args.m} n={args.n} FP64 (seeded U[1,10)/U[100,1000)/U[1,10))",
                   "step": "tableau build (untimed) + first K pivots per seed, oracle on host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{pivs} pivots over {args.steps} steps of {args.m}x{args.n} LPs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2211_10979_gb300 as tsx
    from paper_2211_10979_gb300 import build as tsx_build
    tsx_build.build()
    tsx.use_torch_allocator()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    m, n = args.m, args.n
    seeds = rank_seeds(rank, args.seeds)
    host = {s: lpgen.dense_lp(m, n, s) for s in seeds}
    resident = {s: tuple(torch.from_numpy(v).to(dev) for v in host[s]) for s in seeds}
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    opts = tsx.options(stream=sptr, skip_zero_columns=args.skip_zero, path=args.path,
                       threads=args.threads, blocks=args.blocks)

    x = np.empty(n)
    y = np.empty(m)
    obj = np.empty(1)
    basis = np.empty(m, dtype=np.int32)

    def step(seed):
        dA, db, dc = resident[seed]
        h = tsx.lp_create_device(m, n, dA, db, dc, sptr)
        try:
            st = tsx.lp_solve(h, opts)
            if st != tsx.LP_OPTIMAL:
                raise RuntimeError(f"solve ended {tsx.STATUS_NAMES.get(st, st)}: {tsx.lp_last_error()}")
            tsx.lp_get_solution(h, x, y, obj, basis)
            return tsx.lp_get_stats(h).as_dict()
        finally:
            tsx.lp_destroy(h)

    for k in range(args.warmup):
        step(seeds[k % len(seeds)])
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = [step(seeds[k % len(seeds)]) for k in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    secs = ev0.elapsed_time(ev1) / 1000.0
    pivots = sum(s["iters"] for s in stats)

    # e2e: the public API from pinned host buffers, copies inside the timed region
    pinned = {}
    for s in seeds:
        A, b, c = host[s]
        pinned[s] = tuple(torch.from_numpy(v).pin_memory() for v in (A, b, c))
    xo = torch.empty(n, dtype=torch.float64).pin_memory()
    yo = torch.empty(m, dtype=torch.float64).pin_memory()
    oo = torch.empty(1, dtype=torch.float64).pin_memory()
    bo = torch.empty(m, dtype=torch.int32).pin_memory()

    def e2e_step(seed):
        A, b, c = pinned[seed]
        h = tsx.lp_create(m, n, A, b, c)
        try:
            st = tsx.lp_solve(h, tsx.options(skip_zero_columns=args.skip_zero, path=args.path,
                                             threads=args.threads, blocks=args.blocks))
            if st != tsx.LP_OPTIMAL:
                raise RuntimeError(f"solve ended {tsx.STATUS_NAMES.get(st, st)}")
            _, it = tsx.lp_get_solution(h, xo, yo, oo, bo)
            return it
        finally:
            tsx.lp_destroy(h)

    e2e_piv, e2e_secs = 0, 0.0
    if args.e2e_steps > 0:
        e2e_step(seeds[0])
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_piv = sum(e2e_step(seeds[k % len(seeds)]) for k in range(args.e2e_steps))
        torch.cuda.synchronize(dev)
        e2e_secs = time.perf_counter() - t0

    per_rank = [(pivots, secs, e2e_piv, e2e_secs)]
    if dist:
        t = torch.tensor([pivots, secs, e2e_piv, e2e_secs], dtype=torch.float64, device=dev)
        allt = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(allt, t)
        per_rank = [tuple(v.tolist()) for v in allt]
    value, tmax = combine_ranks([(p, s) for p, s, _, _ in per_rank])
    e2e_value = combine_ranks([(p, s) for _, _, p, s in per_rank])[0] if args.e2e_steps > 0 else None

    if rank == 0:
        peak, peak_src = measured_peaks()
        kernel_ms = sum(s["pivot_ms"] for s in stats) / len(stats)
        upd_bytes = sum(s["update_bytes"] for s in stats) / len(stats)
        dense_bytes = sum(s["dense_update_bytes"] for s in stats) / len(stats)
        achieved = upd_bytes / (kernel_ms / 1000.0) / 1e9
        traffic = profile_traffic(m, n)
        launches = sum(s["kernel_launches"] + 4 for s in stats)   # + validate/reset + 2 extract
        cpu = None
        if not args.no_cpu_baseline:
            cpu = oracle_sample(m, n, seeds[0], args.cpu_seconds)
            cpu.pop("seconds")
            cpu.pop("pivots")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {
                "workload": f"dense LP m={m} n={n} FP64, full solve per step (seeded "
                            "A~U[1,10), b~U[100,1000), c~U[1,10); slack basis; Dantzig)",
                "m": m, "n": n, "seeds_per_rank": len(seeds),
                "pivots_per_step": pivots / args.steps,
                "l2": f"inputs larger than L2 (tableau {(m + 1) * stats[0]['ld'] * 8 / 1e9:.2f} GB)",
                "path": {1: "persistent", 2: "multilaunch"}.get(stats[0]["path"]),
                "grid": stats[0]["grid"], "block": stats[0]["block"],
                "skip_zero_columns": args.skip_zero,
            },
            "roofline": {
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic["bytes_per_launch"] if traffic else None,
                "kernel": "k_pivot_persistent",
                "bytes_per_launch": upd_bytes, "kernel_ms_per_launch": kernel_ms,
                "dense_equivalent_gbs": dense_bytes / (kernel_ms / 1000.0) / 1e9,
                "phase_us_per_pivot": dict(zip(
                    ["ratio", "stage", "update", "wait_ratio", "wait_stage", "wait_update"],
                    [round(1000.0 * sum(st["phase_ms"][k] for st in stats) / max(1, pivots), 3)
                     for k in range(6)])),
            },
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * (m * n + m + n),
                    "d2h_bytes_per_step": 8 * (n + m + 1) + 4 * m},
            "gpu_launches": launches * world,
            "clocks": clk,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if world != args.gpus and world > 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE={world}", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
