"""The multi-rank path of bench.py on CPU: two gloo ranks agree on the slowest replica's time
and the whole-job throughput; the reference arm runs on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [20.0, 25.0][rank]           # rank 1 is the slower replica
        ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
        out[rank] = (ms, bench.job_throughput(world, 4194304, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_throughput():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 25.0
    assert value == pytest.approx(2 * 4194304 / 25e-3 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.job_throughput(1, 1000000, 1000.0) == pytest.approx(1.0)


def test_reference_arm_other_ranks_do_no_work(capsys):
    import argparse

    import bench
    a = argparse.Namespace(kind="sphere", n=1000, mass="loguniform10", theta=0.7, warmup=0, steps=1,
                           cpu_sample_sinks=4)
    bench.run_reference(a, rank=1, world=2)
    assert capsys.readouterr().out == ""
