"""The multi-rank logic of bench.py (independent replicas, weak scaling): the
step time is the maximum over ranks and the rate counts every rank's
particles.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + 5.0 * rank, torch.device("cpu"))
    rate = bench.whole_job_rate(1000, 4, ms, world)
    out[rank] = (ms, rate)
    dist.destroy_process_group()


def test_two_replicas_max_time_and_total_rate():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, rate = res[r]
        assert ms == 15.0  # the slower rank's time
        assert abs(rate - 2 * 1000 * 4 / 0.015) < 1e-6


def test_single_process_is_identity():
    import torch
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_rate(10, 2, 1000.0, 1) == 20.0
