"""The multi-rank path of bench.py: independent replicas, no data-path
collective, the job's rate from the slowest rank (CPU, gloo, world size 2)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    local_solves = [10, 12][rank]
    rate, ms, n = bench.job_rate(local_ms, local_solves)
    reqs = bench.serve_requests(6, seed=5 + rank)
    out[rank] = (rate, ms, n, [k for k, *_ in reqs])
    dist.destroy_process_group()


def test_job_rate_and_sharding_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rate, ms, n, _ = res[r]
        assert ms == 250.0 and n == 22.0
        assert rate == pytest.approx(22.0 / 0.25)
    # each rank serves its own seeded request stream (no shared work)
    assert res[0][3] != res[1][3]


def test_job_rate_single_process():
    import bench
    rate, ms, n = bench.job_rate(50.0, 5)
    assert rate == pytest.approx(100.0) and ms == 50.0 and n == 5
