"""The multi-rank timing of bench.py on CPU: two gloo ranks, max over ranks, whole-job rate."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                  # rank 1 is the slow replica
        worst = bench.max_over_ranks(ms, "cpu")
        out.put((rank, worst, bench.whole_job_rate(1000 * 20, world, worst / 1e3)))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks_and_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, rate in res:
        assert worst == 15.0
        assert rate == pytest.approx(2 * 1000 * 20 / 0.015)


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(100, 1, 2.0) == 50.0


def test_step_kernel_source_hash_is_found():
    # the bench ties a profile's DRAM traffic to the step kernel's source through this hash;
    # it must find the kernel's definition in the source
    import re

    import bench
    h = bench._kernel_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", h)


def test_graph_length_divides_the_timed_steps():
    import bench
    assert bench.graph_length(20, 50) == 20
    assert bench.graph_length(2000, 50) == 50
    assert bench.graph_length(30, 50) == 30
    assert bench.graph_length(120, 50) == 40
    assert bench.graph_length(7, 50) == 7
    assert bench.graph_length(97, 50) == 1
    assert bench.graph_length(100, 0) == 0
