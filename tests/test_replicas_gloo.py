"""Multi-GPU is replicas only: the process group carries no layout data, only
the timing barrier and the max / sum of per-rank timings. These are checked
with two gloo ranks on the CPU (no GPU)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    bench.init_dist("gloo")
    try:
        bench.barrier()
        got = dict(rank=rank,
                   max=bench.max_over_ranks(1.5 + rank),
                   sum=bench.sum_over_ranks(10.0 * (rank + 1)),
                   # rank r processed 100 (r + 1) units in 1000 (r + 1) ms
                   rate=bench.aggregate_rate(100.0 * (rank + 1), 1000.0 * (rank + 1)))
        # the reference arm: ranks other than 0 exit at once without work
        if rank != 0:
            got["ref_rc"] = bench.run_reference(bench_args())
        q.put(got)
        bench.barrier()
    finally:
        dist.destroy_process_group()


def bench_args():
    import argparse
    return argparse.Namespace(config="tiny", warmup=0, steps=1, ref_budget=0.1, gpus=2)


def test_two_gloo_ranks_aggregate_timings():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted((q.get(timeout=5) for _ in range(world)), key=lambda d: d["rank"])
    for d in res:
        assert d["max"] == pytest.approx(2.5)
        assert d["sum"] == pytest.approx(30.0)
        assert d["rate"] == pytest.approx(300.0 / 2.0)
    assert res[1]["ref_rc"] == 0


def test_without_a_process_group_the_values_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.sum_over_ranks(4.0) == 4.0
    assert bench.aggregate_rate(500.0, 250.0) == pytest.approx(2000.0)
