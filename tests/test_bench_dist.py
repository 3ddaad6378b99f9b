"""Host-side logic of the multi-rank benchmark on CPU (gloo, world size 2).

Each rank solves its own LPs (no data-path collective); the job's throughput is
all ranks' pivots over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_rank_seeds_are_disjoint():
    seen = set()
    for r in range(8):
        s = bench.rank_seeds(r, 3)
        assert len(s) == 3 and not (seen & set(s))
        seen |= set(s)
    assert bench.rank_seeds(0, 3) == [1, 2, 3]


def test_combine_takes_the_slowest_rank():
    v, t = bench.combine_ranks([(100, 2.0), (300, 4.0)])
    assert t == 4.0 and v == 100.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pivots, secs = 10.0 * (rank + 1), 1.0 + rank
    t = torch.tensor([pivots, secs], dtype=torch.float64)
    allt = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(allt, t)
    v, tmax = bench.combine_ranks([tuple(a.tolist()) for a in allt])
    q.put((rank, v, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_and_combine_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # ranks: (10 pivots, 1 s), (20 pivots, 2 s) -> 30 pivots / 2 s on both ranks
    assert out == [(0, 15.0, 2.0), (1, 15.0, 2.0)]


def test_reference_arm_other_ranks_exit_without_work(capsys):
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


def test_truncated_fp32_solves_are_refused():
    # the FP32 path finishes a capped float phase with FP64 cleanup pivots, so
    # a pivot cap does not bound its work
    import bench
    with pytest.raises(SystemExit):
        bench.parse_args(["--precision", "fp32", "--max-iters", "5"])
    assert bench.parse_args(["--max-iters", "5"]).max_iters == 5
