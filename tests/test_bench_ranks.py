"""The benchmark's multi-GPU logic is replicas only: each rank times its
own problem, the ranks meet at a barrier, and rank 0 reports the steps of
all ranks over the slowest rank's time.  These run that logic as two gloo
processes on the CPU (no GPU, no NCCL)."""
import json
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        ms_max, value = bench.whole_job(ms, 200, world, "cpu")
        results[rank] = (ms_max, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_and_all_steps():
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_worker, args=(2, port, results), nprocs=2, join=True)
        got = dict(results)
    for rank in (0, 1):
        ms_max, value = got[rank]
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 200 / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.whole_job(40.0, 100, 1, "cpu")
    assert ms_max == 40.0 and value == pytest.approx(2500.0)


def test_reference_arm_prints_only_on_rank_0(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    bench.reference_arm(args)
    assert capsys.readouterr().out == ""
