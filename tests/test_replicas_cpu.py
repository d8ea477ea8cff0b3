"""Host logic of `bench.py --gpus N`: the operator does not shard across GPUs here (replicas only),
so N ranks run independent replicas and the job time is the slowest rank's.  Checked with two gloo
ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (10 + r) ms for the mixed steps and (100 - r) ms for the FP64 steps
        ms = bench.max_over_ranks([10.0 + rank, 100.0 - rank], world, "cpu")
        out[rank] = (ms, bench.job_rate(20, world, ms[0]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == [11.0, 100.0]
        assert rate == pytest.approx(2 * 20 / 0.011)


def test_single_rank_rate():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.job_rate(5, 1, 250.0) == pytest.approx(20.0)
