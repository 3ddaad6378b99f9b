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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 6; batch: 2000, so the timed region spans seconds "
                         "and the clock sampler sees it)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--m", type=int, default=8192)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--seeds", type=int, default=3, help="distinct LPs cycled through the steps")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="solves of the e2e figure (default: as many as the timed steps)")
    ap.add_argument("--skip-zero", type=int, default=1)
    ap.add_argument("--max-iters", type=int, default=-1,
                    help="pivot cap per solve (a truncated solve; default: to the end)")
    ap.add_argument("--device-gen", action="store_true",
                    help="draw the inputs on the device (no e2e, no oracle sample)")
    ap.add_argument("--layout", choices=["condensed", "full"], default="condensed",
                    help="device tableau: nonbasic columns + RHS (condensed) or the whole Table I (full)")
    ap.add_argument("--path", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=0)
    ap.add_argument("--workload", choices=["single", "batch", "serve", "many", "fp64-peak", "hybrid"],
                    default="single",
                    help="batch: 4096 small LPs (m, n uniform in [16, 128]) per step; serve: a "
                         "Poisson stream of LPs (m, n log-uniform in [32, 4096]) through the server")
    ap.add_argument("--thetas", default="1.0,0.995,0.99,0.98,0.95,0.9,0.8",
                    help="hybrid: GPU shares of the column slots to sweep")
    ap.add_argument("--cpu-threads", type=int, default=0, help="hybrid: host threads (0 = all but one)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="serve: length of the stream")
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--plain-seconds", type=float, default=5.0,
                    help="serve: the plain path replays only this much of the stream")
    ap.add_argument("--serve-blocks", type=int, default=0, help="serve: grid cap per single-lane solve")
    ap.add_argument("--serve-team", type=int, default=0,
                    help="serve: blocks per team of the lp_solve_many waves (0 = library default, "
                         "< 0 = no waves: one LP per worker)")
    ap.add_argument("--serve-continuous", type=int, default=1,
                    help="serve: 1 = one continuous team launch for the large requests, 0 = waves")
    ap.add_argument("--serve-path", type=int, default=2,
                    help="serve: single-lane solve path (1 persistent cooperative, 2 one launch per phase)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--many-count", type=int, default=300, help="many: LPs drawn before the size filter")
    ap.add_argument("--many-team", type=int, default=0, help="many: blocks per team (0 = default)")
    ap.add_argument("--batch-threads", type=int, default=0,
                    help="batch: threads per LP (32/64/128/256); 0 = autotuned per size class")
    ap.add_argument("--plain-sample", type=int, default=256,
                    help="LPs of the batch solved one at a time for the plain-path figure")
    ap.add_argument("--generator", choices=["dense", "diag"], default="dense",
                    help="single: lpgen.dense_lp (default) or lpgen.diag_dominant_lp (every "
                         "structural ends basic: a k = m FP64 recovery)")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64",
                    help="fp32: float tableau for every pivot + FP64 recovery on the GPU")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = 2000 if args.workload == "batch" else 6
    if args.e2e_steps < 0:
        args.e2e_steps = 100 if args.workload == "batch" else args.steps
    if args.precision == "fp32" and args.max_iters >= 0:
        # the FP32 path treats a pivot cap as the end of its float phase and
        # lets the FP64 cleanup finish the solve: a truncated FP32 solve is not
        # a fixed amount of work
        ap.error("--max-iters applies to FP64 solves only")
    return args


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


def profile_traffic(m, n, max_iters=-1, layout="condensed", grid=None, block=None):
    """ncu DRAM bytes per launch of the pivot kernel, if a summary for this
    exact kernel build and workload (FP64; a full solve, or the first
    max_iters pivots) is committed under profiles/."""
    path = os.path.join(ROOT, "profiles", "traffic_k_pivot_persistent.txt")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    key = f"{m}x{n}" + (f"@{max_iters}" if max_iters >= 0 else "")
    ent = d.get(key)
    if not ent or ent.get("layout") != layout:
        return None
    from paper_2211_10979_gb300 import build as b
    if ent.get("source_digest") != b.source_digest(b.PIVOT_SOURCES):
        return None   # the kernel changed since the counters were taken
    if (grid, block) != (ent.get("grid", grid), ent.get("block", block)):
        return None   # another launch shape
    return ent


def host_cpu():
    """The host's CPU model (lscpu, else /proc/cpuinfo) and its core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


class pinned_to_one_core:
    """Runs the block with the process pinned to one core (the last one the
    process may use), then restores the previous affinity."""

    def __enter__(self):
        self.prev = None
        try:
            self.prev = os.sched_getaffinity(0)
            self.core = max(self.prev)
            os.sched_setaffinity(0, {self.core})
        except (AttributeError, OSError):
            self.core = None
        return self

    def __exit__(self, *exc):
        if self.prev is not None:
            try:
                os.sched_setaffinity(0, self.prev)
            except OSError:
                pass


def oracle_sample(m, n, seed, budget_s):
    """The CPU oracle on a bounded sample of the workload: the tableau build and
    the first K pivots of the same LP, K chosen so the pivots take ~budget_s,
    on one core (the process pinned to it)."""
    with pinned_to_one_core() as pin:
        r = _oracle_sample(m, n, seed, budget_s)
    r.update(host_cpu())
    r["pinned_core"] = pin.core
    return r


def _oracle_sample(m, n, seed, budget_s):
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
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": f"{pivs} pivots over {args.steps} steps of {args.m}x{args.n} LPs, "
                                        "the process pinned to one core"}, **host_cpu()),
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
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    if args.device_gen:   # inputs drawn on the device (sizes whose A does not fit host memory)
        host = {}
        resident = {}
        for s in seeds:
            dA = torch.empty(m * n, dtype=torch.float64, device=dev)
            db = torch.empty(m, dtype=torch.float64, device=dev)
            dc = torch.empty(n, dtype=torch.float64, device=dev)
            tsx.lp_generate_dense(m, n, s, dA, db, dc, sptr)
            resident[s] = (dA, db, dc)
        torch.cuda.synchronize(dev)
        args.e2e_steps = 0
        args.no_cpu_baseline = True
    else:
        gen = lpgen.diag_dominant_lp if args.generator == "diag" else lpgen.dense_lp
        host = {s: gen(m, n, s) for s in seeds}
        resident = {s: tuple(torch.from_numpy(v).to(dev) for v in host[s]) for s in seeds}
    prec = tsx.LP_PREC_FP32 if args.precision == "fp32" else tsx.LP_PREC_FP64
    layout = tsx.LP_LAYOUT_FULL if args.layout == "full" else tsx.LP_LAYOUT_CONDENSED
    opts = tsx.options(stream=sptr, skip_zero_columns=args.skip_zero, path=args.path,
                       threads=args.threads, blocks=args.blocks, precision=prec, layout=layout,
                       max_iters=args.max_iters)
    done_ok = (tsx.LP_OPTIMAL, tsx.LP_ITER_LIMIT) if args.max_iters >= 0 else (tsx.LP_OPTIMAL,)

    x = np.empty(n)
    y = np.empty(m)
    obj = np.empty(1)
    basis = np.empty(m, dtype=np.int32)

    def step(seed):
        dA, db, dc = resident[seed]
        h = tsx.lp_create_device(m, n, dA, db, dc, sptr)
        try:
            st = tsx.lp_solve(h, opts)
            if st not in done_ok:
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
    for s in seeds if args.e2e_steps > 0 else ():
        A, b, c = host[s]
        pinned[s] = tuple(torch.from_numpy(v).pin_memory() for v in (A, b, c))
    xo = torch.empty(n, dtype=torch.float64).pin_memory()
    yo = torch.empty(m, dtype=torch.float64).pin_memory()
    oo = torch.empty(1, dtype=torch.float64).pin_memory()
    bo = torch.empty(m, dtype=torch.int32).pin_memory()

    split = {"create_h2d_s": 0.0, "solve_s": 0.0, "readout_d2h_s": 0.0, "destroy_s": 0.0}
    create_dev = {"copy_ms": [], "check_ms": [], "wall_ms": []}   # lp_create's own timings, per step

    def e2e_step(seed):
        A, b, c = pinned[seed]
        t0 = time.perf_counter()
        h = tsx.lp_create(m, n, A, b, c)      # H2D of A, b, c and the input check
        t1 = time.perf_counter()
        try:
            st = tsx.lp_solve(h, tsx.options(skip_zero_columns=args.skip_zero, path=args.path,
                                             threads=args.threads, blocks=args.blocks,
                                             precision=prec, layout=layout))
            t2 = time.perf_counter()
            if st != tsx.LP_OPTIMAL:
                raise RuntimeError(f"solve ended {tsx.STATUS_NAMES.get(st, st)}")
            _, it = tsx.lp_get_solution(h, xo, yo, oo, bo)
            t3 = time.perf_counter()
            cs = tsx.lp_get_stats(h)
            create_dev["copy_ms"].append(cs.create_copy_ms)
            create_dev["check_ms"].append(cs.create_check_ms)
            create_dev["wall_ms"].append(cs.create_wall_ms)
        finally:
            tsx.lp_destroy(h)
        t4 = time.perf_counter()
        split["create_h2d_s"] += t1 - t0
        split["solve_s"] += t2 - t1
        split["readout_d2h_s"] += t3 - t2
        split["destroy_s"] += t4 - t3
        return it

    e2e_piv, e2e_secs = 0, 0.0
    if args.e2e_steps > 0:
        e2e_step(seeds[0])
        # warm-up: one upload from every pinned buffer (the GPU's first read of
        # a pinned buffer maps it and runs at ~50 GB/s; later reads at the
        # link's ~210 GB/s), untimed
        for s_ in seeds[1:]:
            tsx.lp_destroy(tsx.lp_create(m, n, *pinned[s_]))
        for k in split:
            split[k] = 0.0
        for v in create_dev.values():
            v.clear()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_piv = sum(e2e_step(seeds[k % len(seeds)]) for k in range(args.e2e_steps))
        torch.cuda.synchronize(dev)
        e2e_secs = time.perf_counter() - t0

    # FP32 path: objective error of each timed seed against the FP64 path
    # (untimed), which equals the FP64 oracle step by step
    prec_info = None
    if args.precision == "fp32" and args.max_iters < 0:
        errs = []
        for sd in seeds:
            dA, db, dc = resident[sd]
            h = tsx.lp_create_device(m, n, dA, db, dc, sptr)
            try:
                tsx.lp_solve(h, tsx.options(stream=sptr, precision=tsx.LP_PREC_FP32))
                o32 = np.empty(1)
                tsx.lp_get_solution(h, None, None, o32, None)
                s32 = tsx.lp_get_stats(h).as_dict()
                tsx.lp_solve(h, tsx.options(stream=sptr))
                o64 = np.empty(1)
                tsx.lp_get_solution(h, None, None, o64, None)
                errs.append((abs(o32[0] - o64[0]) / abs(o64[0]), s32))
            finally:
                tsx.lp_destroy(h)
        prec_info = {
            "objective_rel_err_vs_fp64_max": max(e for e, _ in errs),
            "cleanup_pivots": [st_["cleanup_pivots"] for _, st_ in errs],
            "k": [st_["k"] for _, st_ in errs],
            "recover_ms": [round(st_["recover_ms"], 3) for _, st_ in errs],
            "primal_violation_max": max(st_["primal_violation"] for _, st_ in errs),
            "dual_violation_max": max(st_["dual_violation"] for _, st_ in errs),
        }

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
        traffic = profile_traffic(m, n, args.max_iters, args.layout, stats[0]["grid"], stats[0]["block"])
        launches = sum(s["kernel_launches"] + 4 for s in stats)   # + validate/reset + 2 extract
        cpu = None
        if not args.no_cpu_baseline:
            cpu = oracle_sample(m, n, seeds[0], args.cpu_seconds)
            cpu.pop("seconds")
            cpu.pop("pivots")
        elem = 4 if args.precision == "fp32" else 8
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32 tableau + f64 recovery",
            "data": "synthetic",
            "config": {
                "workload": f"dense LP m={m} n={n} {args.precision.upper()}, "
                            + ("full solve" if args.max_iters < 0 else f"first {args.max_iters} pivots")
                            + (" per step (seeded A~U[1,10), b~U[100,1000), c~U[1,10); slack basis; Dantzig)"
                               if args.generator == "dense" else
                               " per step (seeded diagonally dominant A: A_ij~U[0,1), A_ii+=4max(m,n); "
                               "b~U[100,1000), c~U[1,10); every structural ends basic)"),
                "m": m, "n": n, "seeds_per_rank": len(seeds),
                "pivots_per_step": pivots / args.steps,
                "l2": f"inputs larger than L2 (tableau {(m + 1) * stats[0]['ld'] * elem / 1e9:.2f} GB)",
                "layout": args.layout,
                "path": {1: "persistent", 2: "multilaunch", 4: "cluster"}.get(stats[0]["path"]),
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
                    "d2h_bytes_per_step": 8 * (n + m + 1) + 4 * m,
                    "steps": args.e2e_steps,
                    "ms_per_step": {k.replace("_s", "_ms"): round(1e3 * v / max(1, args.e2e_steps), 3)
                                    for k, v in split.items()},
                    "create_ms_by_step": {k: [round(x, 3) for x in v] for k, v in create_dev.items()},
                    "what": "wall time per solve through the public API from pinned host buffers: "
                            "lp_create (H2D + input check), lp_solve, lp_get_solution (D2H), "
                            "lp_destroy; create_ms_by_step: lp_create's own device times of the "
                            "copy and the check (CUDA events) and host time of the call"},
            "gpu_launches": launches * world,
            "clocks": clk,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if prec_info:
            line["precision"] = prec_info
            line["roofline"]["traffic"] = None
        if stats[0]["path"] == 4:
            # the cluster path keeps the tableau on chip: its ceiling is the
            # FP64 pipes of the cluster's SMs, not HBM
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            csize = stats[0]["grid"]
            peak_all, probe = fp64_fma_rate(tsx, sptr)
            peak_c = peak_all * csize / nsm
            flops = 2.0 * (m + 1) * (n + 1) * pivots / args.steps   # one fma per condensed entry
            ach = flops / (kernel_ms / 1000.0) / 1e12
            line["roofline"] = {
                "bound": "alu", "achieved": ach, "peak": peak_c, "unit": "TFLOP/s", "frac": ach / peak_c,
                "peak_source": f"measured FP64 fma rate of the whole GPU in this run ({peak_all:.3f} TFLOP/s, "
                               f"lp_measure_fp64_fma_rate) x {csize}/{nsm} SMs of one cluster",
                "frac_of_whole_gpu": ach / peak_all, "probe": probe, "traffic": None,
                "kernel": "k_cluster_solve", "cluster_blocks": csize,
                "flops_per_launch": flops, "kernel_ms_per_launch": kernel_ms,
                "us_per_pivot": 1000.0 * kernel_ms * args.steps / max(1, pivots),
                "phase_us_per_pivot": dict(zip(
                    ["step2", "wait_barrier1", "minimum_and_R", "wait_barrier2", "step3", "step1"],
                    [round(1000.0 * sum(st["phase_ms"][k] for st in stats) / max(1, pivots), 3)
                     for k in range(6)])),
            }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


FP64_PEAK_TFLOPS = 1.25   # GB300 nominal FP64 (one DFMA = 2 flops)


def fp64_fma_rate(tsx, sptr, seconds=0.5, repeats=3):
    """Measured FP64 ceiling: the best of `repeats` launches of the library's
    DFMA-chain probe (lp_measure_fp64_fma_rate), each sized to ~`seconds`;
    returns (TFLOP/s at 2 flops per fma, details)."""
    from paper_2211_10979_gb300 import abi
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    blocks, threads = props.multi_processor_count * 8, 256
    ms, rate = abi.lp_measure_fp64_fma_rate(blocks, threads, 1000, sptr)
    iters = max(1000, int(1000 * seconds / max(ms * 1e-3, 1e-6)))
    best = 0.0
    for _ in range(repeats):
        ms, rate = abi.lp_measure_fp64_fma_rate(blocks, threads, iters, sptr)
        best = max(best, rate)
    return 2.0 * best / 1e12, {"blocks": blocks, "threads": threads, "chains": 8,
                                "iters": iters, "launch_ms": ms}


def run_fp64_peak(args, rank, world, local):
    """The FP64 pipe's measured ceiling (DFMA chains), with the clock record."""
    import torch
    torch.cuda.set_device(local)
    import paper_2211_10979_gb300 as tsx
    from paper_2211_10979_gb300 import build as tsx_build
    tsx_build.build()
    sptr = torch.cuda.current_stream().cuda_stream
    fp64_fma_rate(tsx, sptr, seconds=0.2, repeats=args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    tflops, info = fp64_fma_rate(tsx, sptr, seconds=1.0, repeats=max(1, args.steps))
    # how the pipe charges partial warps and divisions (warp instructions/s)
    from paper_2211_10979_gb300 import abi
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    blocks = props.multi_processor_count * 8
    charge = {}
    for op, name, iters in ((0, "fma", 20000), (1, "div", 2000)):
        for lanes in (32, 16, 1):
            abi.lp_measure_fp64_op_rate(op, lanes, blocks, 256, iters // 10, sptr)
            ms, wps = abi.lp_measure_fp64_op_rate(op, lanes, blocks, 256, iters, sptr)
            charge[f"{name}_lanes{lanes}_warp_instr_per_s"] = wps
    charge["div_cost_in_fma"] = charge["fma_lanes32_warp_instr_per_s"] / charge["div_lanes32_warp_instr_per_s"]
    clk = clocks.stop()
    if rank == 0:
        print(json.dumps({"metric": "FP64 fma rate", "value": tflops, "unit": "TFLOP/s",
                          "fma_per_s": tflops * 1e12 / 2.0, "n_gpus": 1, "probe": info,
                          "nominal_tflops": FP64_PEAK_TFLOPS, "frac_of_nominal": tflops / FP64_PEAK_TFLOPS,
                          "pipe_charge": charge, "clocks": clk}), flush=True)
    return 0


def batch_problems(count, seed):
    """The batching workload: LP k has m, n uniform in [16, 128] and the dense
    generator's data with seed 10_000 + k (per-rank offsets by `seed`)."""
    shapes = lpgen.batch_shapes(count, 16, 128, seed)
    return [lpgen.dense_lp(mm, nn, 10_000 * seed + k) for k, (mm, nn) in enumerate(shapes)]


def oracle_batch_sample(problems, budget_s):
    import oracle
    with pinned_to_one_core() as pin:
        t0 = time.perf_counter()
        done = 0
        for A, b, c in problems:
            oracle.solve(A, b, c, log_cap=1)
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        secs = time.perf_counter() - t0
    return dict({"value": done / secs, "unit": "LPs/s", "cores": 1, "kind": "oracle",
                 "sample": f"first {done} LPs of the batch, solved one by one (single-threaded C, FP64)",
                 "pinned_core": pin.core}, **host_cpu())


def run_batch(args, rank, world, local):
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
    count = args.batch_count
    problems = batch_problems(count, 1 + rank)
    m = np.array([p[0].shape[0] for p in problems], dtype=np.int32)
    n = np.array([p[0].shape[1] for p in problems], dtype=np.int32)
    A = np.concatenate([p[0].ravel() for p in problems])
    b = np.concatenate([p[1] for p in problems])
    c = np.concatenate([p[2] for p in problems])
    dA, db, dc = (torch.from_numpy(v).to(dev) for v in (A, b, c))
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    status = np.empty(count, dtype=np.int32)
    iters = np.empty(count, dtype=np.int64)
    obj = np.empty(count)
    x = np.empty(int(n.sum()))
    y = np.empty(int(m.sum()))
    h = tsx.lp_batch_create_device(count, m, n, dA, db, dc, sptr)
    opts = tsx.batch_options(stream=sptr, threads=args.batch_threads)
    try:
        for _ in range(args.warmup):   # the first solve autotunes and captures the graph
            tsx.lp_batch_solve(h, opts)
            tsx.lp_batch_get(h, status, iters, obj, x, y)
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(local) if rank == 0 else None
        if clocks:
            clocks.start()
        if dist:
            dist.barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        kernel_ms = 0.0
        for _ in range(args.steps):
            if tsx.lp_batch_solve(h, opts) != 0:
                raise RuntimeError(tsx.lp_last_error())
            tsx.lp_batch_get(h, status, iters, obj, x, y)
            kernel_ms += tsx.lp_batch_get_stats(h).solve_ms
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        secs = ev0.elapsed_time(ev1) / 1000.0
        bstats = tsx.lp_batch_get_stats(h).as_dict()
    finally:
        tsx.lp_batch_destroy(h)
    assert (status == 0).all(), "every LP of the workload is solved to optimality"
    fp64_peak, fp64_probe = fp64_fma_rate(tsx, sptr)
    pivots = int(iters.sum())
    flops = float(np.sum(2.0 * (m + 1.0) * (n + 1.0) * iters))   # one FMA per condensed entry

    # plain path: the same resident LPs one at a time through lp_create_device / lp_solve
    k_plain = min(args.plain_sample, count)
    offs_a = np.concatenate([[0], np.cumsum(m.astype(np.int64) * n)])
    offs_b = np.concatenate([[0], np.cumsum(m)])
    offs_c = np.concatenate([[0], np.cumsum(n)])
    xo = np.empty(int(n.max()))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(k_plain):
        hk = tsx.lp_create_device(int(m[k]), int(n[k]), dA[offs_a[k]:offs_a[k + 1]], db[offs_b[k]:offs_b[k + 1]],
                                  dc[offs_c[k]:offs_c[k + 1]], sptr)
        try:
            tsx.lp_solve(hk, tsx.options(stream=sptr))
            tsx.lp_get_solution(hk, xo[:n[k]], None, None, None)
        finally:
            tsx.lp_destroy(hk)
    plain_secs = time.perf_counter() - t0

    # e2e: packed inputs from pinned host memory, copies inside the timed region
    pA, pb, pc = (torch.from_numpy(v).pin_memory() for v in (A, b, c))
    e2e_steps = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        he = tsx.lp_batch_create(count, m, n, pA, pb, pc)
        try:
            tsx.lp_batch_solve(he, tsx.batch_options())   # reuses the device's tuned threads
            tsx.lp_batch_get(he, status, iters, obj, x, y)
        finally:
            tsx.lp_batch_destroy(he)
    e2e_secs = time.perf_counter() - t0

    per_rank = [(count * args.steps, secs, count * e2e_steps, e2e_secs)]
    if dist:
        t = torch.tensor(per_rank[0], dtype=torch.float64, device=dev)
        allt = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(allt, t)
        per_rank = [tuple(v.tolist()) for v in allt]
    value, tmax = combine_ranks([(p, s_) for p, s_, _, _ in per_rank])
    e2e_value, _ = combine_ranks([(p, s_) for _, _, p, s_ in per_rank])
    if rank == 0:
        kernel_s = kernel_ms / 1000.0 / args.steps
        achieved = flops / kernel_s / 1e12
        line = {
            "metric": "LPs/s", "value": value, "unit": "LPs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"batch of {count} dense LPs, m and n uniform in [16, 128], FP64, "
                                   "one solve of the whole batch per step (results copied to the host)",
                       "pivots_per_step": pivots, "classes": bstats["lps_per_class"],
                       "threads_per_lp": bstats["threads"], "graph": bstats["graph"],
                       "l2": f"inputs {A.nbytes / 1e6:.0f} MB; tableaux in shared memory"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak,
                         "peak_source": "measured in this run: the library's DFMA-chain probe "
                                        "(lp_measure_fp64_fma_rate, best of 3 launches of ~0.5 s, "
                                        "2 flops per fma)",
                         "probe": fp64_probe, "frac_of_nominal": achieved / FP64_PEAK_TFLOPS,
                         "traffic": None, "kernel": "k_batch_solve",
                         "flops_per_launch": flops, "kernel_ms_per_launch": 1000.0 * kernel_s,
                         "pivots_per_s": pivots / kernel_s},
            "plain": {"value": k_plain / plain_secs, "unit": "LPs/s",
                      "sample": f"first {k_plain} LPs of the batch, lp_create_device + lp_solve + "
                                "lp_get_solution one at a time",
                      "speedup_of_batch": value / (k_plain / plain_secs)},
            "e2e": {"value": e2e_value, "unit": "LPs/s", "h2d_bytes_per_step": int(A.nbytes + b.nbytes + c.nbytes),
                    "d2h_bytes_per_step": int(status.nbytes + iters.nbytes + obj.nbytes + x.nbytes + y.nbytes)},
            "gpu_launches": int(bstats["kernel_launches"]) * args.steps * world,
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_batch_sample(problems, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def many_shapes(count, seed):
    """The LPs of the serving distribution (m, n log-uniform in [32, 4096])
    whose condensed FP64 tableau exceeds one SM's shared memory: the ones the
    server solves in lp_solve_many waves."""
    shapes = lpgen.loguniform_shapes(count, 32, 4096, seed)
    return [(m, n) for m, n in shapes if (m + 1) * (n + 2) * 8 > 232_448]


def run_many(args, rank, world, local):
    """lp_solve_many on the medium and large LPs of the serving distribution,
    inputs resident in HBM; plain = the same LPs one at a time by lp_solve."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2211_10979_gb300 as tsx
    from paper_2211_10979_gb300 import build as tsx_build
    tsx_build.build()
    tsx.use_torch_allocator()
    shapes = many_shapes(args.many_count, 5 + rank)
    seeds = [1000 + k for k in range(len(shapes))]
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    prec = tsx.LP_PREC_FP32 if args.precision == "fp32" else tsx.LP_PREC_FP64
    inputs = []
    for (m, n), sd in zip(shapes, seeds):
        dA = torch.empty(m * n, dtype=torch.float64, device=dev)
        db = torch.empty(m, dtype=torch.float64, device=dev)
        dc = torch.empty(n, dtype=torch.float64, device=dev)
        tsx.lp_generate_dense(m, n, sd, dA, db, dc, sptr)
        inputs.append((dA.view(m, n), db, dc))
    torch.cuda.synchronize(dev)
    prs = [tsx.Problem(dA, db, dc, device=True, stream=sptr) for dA, db, dc in inputs]
    opts = tsx.options(precision=prec, blocks=args.many_team, stream=sptr)
    for _ in range(args.warmup):
        tsx.solve_many(prs, opts)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    walls, kernel_ms, upd = [], [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = tsx.solve_many(prs, opts)
        walls.append(time.perf_counter() - t0)
        stats = [pr.stats() for pr in prs]
        kernel_ms.append(stats[0]["pivot_ms"])
        upd.append(sum(x["update_bytes"] for x in stats))
    clk = clocks.stop()
    bad = sum(1 for v in st if v != tsx.LP_OPTIMAL)
    pivots = sum(x["iters"] for x in stats)
    value = len(prs) * args.steps / sum(walls)
    k_ms = statistics.median(kernel_ms)
    achieved = statistics.median(upd) / (k_ms / 1000.0) / 1e9
    peak, peak_src = measured_peaks()
    # plain: every LP once through lp_solve (default persistent path)
    po = tsx.options(precision=prec, stream=sptr)
    t0 = time.perf_counter()
    for pr in prs:
        pr.solve(po)
    plain = len(prs) / (time.perf_counter() - t0)
    # e2e: pinned host inputs, handles created and results read back inside the timed region
    pinned = [tuple(t.cpu().pin_memory() for t in inp) for inp in inputs]
    host = [tuple(t.numpy() for t in tp) for tp in pinned]   # views of the pinned buffers
    e2e_steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hp = [tsx.Problem(A, b, c) for A, b, c in host]
        tsx.solve_many(hp, opts)
        for pr in hp:
            pr.solution()
            pr.close()
    e2e = len(prs) * e2e_steps / (time.perf_counter() - t0)
    for pr in prs:
        pr.close()
    cpu = None if args.no_cpu_baseline else oracle_batch_sample(host, args.cpu_seconds)
    line = {
        "metric": "LPs/s", "value": value, "unit": "LPs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * sum(walls) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 tableau + f64 recovery" if prec == tsx.LP_PREC_FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": f"lp_solve_many over the {len(prs)} LPs of {args.many_count} drawn from the "
                               "serving distribution (m, n log-uniform in [32, 4096]) whose condensed tableau "
                               "exceeds one SM's shared memory; one call per step, inputs resident in HBM",
                   "team_blocks": args.many_team or 16, "pivots_per_step": pivots,
                   "l2": "tableaux of the step total well above L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)", "traffic": None,
                     "kernel": "k_team_solve", "kernel_ms_per_launch": k_ms,
                     "bytes_per_launch": statistics.median(upd)},
        "plain": {"value": plain, "unit": "LPs/s", "path": "the same LPs one at a time through lp_solve",
                  "speedup": value / plain},
        "non_optimal": bad,
        "e2e": {"value": e2e, "unit": "LPs/s",
                "h2d_bytes_per_step": int(sum(8 * (m * n + m + n) for m, n in shapes)),
                "d2h_bytes_per_step": int(sum(8 * (m + n + 1) for m, n in shapes)),
                "note": "lp_create from pinned host arrays, lp_solve_many, lp_get_solution, lp_destroy"},
        "gpu_launches": int(sum(x["kernel_launches"] for x in stats)) * args.steps,
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def play_stream(tsx, torch, dev, shapes, arrivals, seeds, server_kw):
    """Submits each request at its arrival time (inputs generated on the device
    just before), collects every result, returns per-request (status, latency
    s, obj, done time) in submission order and the server's statistics.
    Latency runs from the scheduled arrival.  The inputs of finished requests
    are released during the stream (a long stream does not keep them all)."""
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    out = [None] * len(shapes)
    with tsx.Server(**server_kw) as sv:
        pending = {}
        last_sweep = time.monotonic()

        def sweep(block):
            for ticket in list(pending):
                if not block and sv.wait(ticket, 0.0) == tsx.LP_PENDING:
                    continue
                sv.wait(ticket)
                idx, t_sched, _ = pending.pop(ticket)
                r = sv.result(ticket)
                out[idx] = (r.status, r.t_done - t_sched, r.obj, r.t_done)

        t0 = time.monotonic()
        for idx, ((m, n), t_arr, sd) in enumerate(zip(shapes, arrivals, seeds)):
            delay = t0 + t_arr - time.monotonic()
            if delay > 0:
                time.sleep(delay)
            dA = torch.empty(m * n, dtype=torch.float64, device=dev)
            db = torch.empty(m, dtype=torch.float64, device=dev)
            dc = torch.empty(n, dtype=torch.float64, device=dev)
            tsx.lp_generate_dense(m, n, sd, dA, db, dc, sptr)
            stream.synchronize()
            pending[sv.submit_device(m, n, dA, db, dc)] = (idx, t0 + t_arr, (dA, db, dc))
            if time.monotonic() - last_sweep > 0.02:
                sweep(False)
                last_sweep = time.monotonic()
        sweep(True)
        st = sv.stats()
        st["last_error"] = sv.last_error()
    return out, st, t0


def run_serve(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2211_10979_gb300 as tsx
    from paper_2211_10979_gb300 import build as tsx_build
    tsx_build.build()
    count = max(1, int(args.rate * args.serve_seconds))
    seed = 5 + rank
    arrivals = lpgen.poisson_arrivals(count, args.rate, seed)
    shapes = lpgen.loguniform_shapes(count, 32, 4096, seed)
    seeds = [100_000 * seed + k for k in range(count)]
    # warm-up: tune the batched solver and load every kernel once
    play_stream(tsx, torch, dev, shapes[:64], arrivals[:64] * 0.0, seeds[:64], {"workers": 4})
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    served, st, t0 = play_stream(tsx, torch, dev, shapes, arrivals, seeds,
                                 {"workers": args.serve_workers, "blocks_per_lp": args.serve_blocks,
                                  "path": args.serve_path, "team_blocks": args.serve_team,
                                  "continuous": args.serve_continuous})
    clk = clocks.stop()
    # the plain path on the stream's first plain_seconds (it cannot keep up
    # with the arrival rate: its queue grows along the whole stream)
    kp = max(1, min(count, int(np.searchsorted(arrivals, args.plain_seconds))))
    plain, st_plain, t0p = play_stream(tsx, torch, dev, shapes[:kp], arrivals[:kp], seeds[:kp],
                                       {"workers": 1, "batch_small": 0, "path": 0, "team_blocks": -1})

    def summary(res, t_start):
        lat = np.array([r[1] for r in res])
        t_end = max(r[3] for r in res)
        ok = sum(1 for r in res if r[0] == 0)
        return {"solves_per_s": len(res) / (t_end - t_start), "optimal": ok,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}

    s_srv = summary(served, t0)
    s_pl = summary(plain, t0p)
    hist = {}
    for r in served:
        hist[tsx.STATUS_NAMES.get(r[0], str(r[0]))] = hist.get(tsx.STATUS_NAMES.get(r[0], str(r[0])), 0) + 1
    rel = [abs(a[2] - b[2]) / max(1e-300, abs(b[2])) for a, b in zip(served[:kp], plain)]
    line = {
        "metric": "LPs/s", "value": s_srv["solves_per_s"], "unit": "LPs/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * count / s_srv["solves_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 micro-batches (LPs whose condensed tableau fits one SM's shared memory); "
                 "f32 tableau + f64 recovery in lp_solve_many waves (the others)",
        "data": "synthetic",
        "config": {"workload": f"Poisson stream, {args.rate:.0f} LPs/s for {args.serve_seconds:.1f} s "
                               f"({count} LPs), m and n log-uniform in [32, 4096], inputs generated on "
                               "the device at arrival; continuous batching, 64 GiB admission budget",
                   "workers": args.serve_workers, "blocks_per_lp": args.serve_blocks or "default",
                   "single_lane_path": args.serve_path,
                   "batches": st["batches"], "batched_lps": st["batched_lps"],
                   "large_lane": "continuous team launch" if args.serve_continuous else "lp_solve_many waves",
                   "lane_lps": st["lane_lps"], "lane_launches": st["lane_launches"],
                   "waves": st["waves"], "wave_lps": st["wave_lps"], "team_blocks": args.serve_team or "default",
                   "wave_ms": round(st["wave_ms"], 1), "wave_kernel_ms": round(st["wave_kernel_ms"], 1),
                   "wave_create_ms": round(st["wave_create_ms"], 1), "wave_wait_ms": round(st["wave_wait_ms"], 1),
                   "wave_launch_ms": round(st["wave_launch_ms"], 1),
                   "peak_admitted_bytes": st["peak_bytes"]},
        "latency": {"p50_ms": s_srv["p50_ms"], "p99_ms": s_srv["p99_ms"], "mean_ms": s_srv["mean_ms"],
                    "max_ms": s_srv["max_ms"], "from": "scheduled arrival to result on the host",
                    "breakdown_ms": {
                        "queue": [round(st["queue_p50_ms"], 2), round(st["queue_p99_ms"], 2)],
                        "wait_for_launch": [round(st["wait_p50_ms"], 2), round(st["wait_p99_ms"], 2)],
                        "kernel": [round(st["run_p50_ms"], 2), round(st["run_p99_ms"], 2)],
                        "recovery_readout": [round(st["post_p50_ms"], 2), round(st["post_p99_ms"], 2)],
                        "server_total": [round(st["lat_p50_ms"], 2), round(st["lat_p99_ms"], 2)],
                        "what": "[p50, p99] per stage, measured in the server: submit -> admitted by a "
                                "worker -> its launch starts (a wave waits for the previous wave's launch) "
                                "-> its kernel completes (a wave: the whole team launch) -> result stored"}},
        "plain": dict(s_pl, path="one LP at a time in arrival order (1 worker, no micro-batches)",
                      sample=f"the stream's first {kp} requests ({args.plain_seconds:g} s of arrivals)"),
        "speedup_vs_plain": s_srv["solves_per_s"] / s_pl["solves_per_s"],
        "objective_rel_diff_vs_plain_max": max(rel),
        "optimal": s_srv["optimal"], "status_counts": hist, "last_error": st["last_error"] or None,
        "e2e": {"value": s_srv["solves_per_s"], "unit": "LPs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(sum(8 * (m + n + 1) for m, n in shapes)),
                "note": "inputs are generated on the device at each arrival; results copied to the host"},
        "roofline": None,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_hybrid(args, rank, world, local):
    """The paper's CPU+GPU column split (Section IV; Tables VI-VIII): one whole
    solve of the seed-1 LP per share theta of the column slots on the GPU, the
    rest on host threads, beside the GPU-only persistent path.  Context, not a
    target: wall-clock time of lp_solve (host threads and GPU kernel alike)."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2211_10979_gb300 as tsx
    from paper_2211_10979_gb300 import build as tsx_build
    tsx_build.build()
    tsx.use_torch_allocator()
    m, n = args.m, args.n
    A, b, c = lpgen.dense_lp(m, n, 1)
    dA, db, dc = (torch.from_numpy(v).to(dev) for v in (A, b, c))
    sptr = torch.cuda.current_stream(dev).cuda_stream
    rows = []
    with tsx.Problem(dA, db, dc, device=True, stream=sptr) as pr:
        def timed(**kw):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            st = pr.solve(tsx.options(stream=sptr, **kw))
            secs = time.perf_counter() - t0
            if st != tsx.LP_OPTIMAL:
                raise RuntimeError(f"solve ended {tsx.STATUS_NAMES.get(st, st)}: {tsx.lp_last_error()}")
            sol = pr.solution()
            return secs, sol.iters, sol.obj
        for _ in range(max(1, args.warmup)):
            timed(path=tsx.LP_PATH_PERSISTENT)
        clocks = ClockSampler(local)
        clocks.start()
        base_s, base_it, base_obj = min((timed(path=tsx.LP_PATH_PERSISTENT) for _ in range(args.steps)),
                                        key=lambda r: r[0])
        rows.append({"theta": "GPU only (persistent path)", "seconds": base_s, "pivots": base_it,
                     "pivots_per_s": base_it / base_s, "vs_gpu_only": 1.0})
        for th in [float(x) for x in args.thetas.split(",") if x]:
            timed(path=tsx.LP_PATH_HYBRID, gpu_share=th, cpu_threads=args.cpu_threads)   # warm-up
            secs, it, obj = min((timed(path=tsx.LP_PATH_HYBRID, gpu_share=th, cpu_threads=args.cpu_threads)
                                 for _ in range(args.steps)), key=lambda r: r[0])
            assert it == base_it and obj == base_obj, "the split changes no pivot"
            rows.append({"theta": th, "seconds": secs, "pivots": it, "pivots_per_s": it / secs,
                         "vs_gpu_only": base_s / secs})
        clk = clocks.stop()
    hw = os.cpu_count()
    line = {
        "metric": "pivots/s", "value": rows[0]["pivots_per_s"], "unit": "pivots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"dense LP m={m} n={n} FP64 seed 1, whole solve per theta (best of {args.steps})",
                   "what": "theta = share of the nonbasic column slots on the GPU; the rest on host threads "
                           "(the paper's Section IV split); wall-clock time of lp_solve",
                   "cpu_threads": args.cpu_threads or max(1, hw - 1), "host_cores": hw},
        "sweep": rows, "clocks": clk, "roofline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if world != args.gpus and world > 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE={world}", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world, local)
    if args.workload == "fp64-peak":
        return run_fp64_peak(args, rank, world, local) if rank == 0 else 0
    if args.workload == "hybrid":
        return run_hybrid(args, rank, world, local) if rank == 0 else 0
    if args.workload == "many":
        if rank != 0:
            return 0
        return run_many(args, rank, world, local)
    if args.workload == "serve":
        if rank != 0:
            return 0
        return run_serve(args, rank, world, local)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
