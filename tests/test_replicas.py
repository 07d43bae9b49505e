"""Replica timing on two gloo ranks (CPU): the job time is the slowest rank's
and the job throughput counts every rank's operations."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_2407_13055_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.barrier()
        ms = 10.0 * (rank + 1)          # rank r "took" 10 (r + 1) ms
        ms_max = replicas.max_over_ranks(ms)
        out[rank] = (replicas.world_size(), ms_max, replicas.job_throughput(32, ms_max, world))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_sum_the_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(2):
        world, ms_max, thr = res[r]
        assert world == 2 and ms_max == 20.0
        assert thr == pytest.approx(2 * 32 / 0.020)


def test_single_process_is_identity():
    from paper_2407_13055_gb300 import replicas
    assert replicas.world_size() == 1
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10, 1000.0, 1) == 10.0
    with pytest.raises(ValueError):
        replicas.job_throughput(1, 0.0, 1)
