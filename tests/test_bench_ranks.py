"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each a replica;
the job time is the slowest rank's and the throughput counts every rank's bytes."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 + 50.0 * rank                      # rank 1 is the slow replica
    mx = bench.max_over_ranks(my_ms, world)
    out[rank] = (mx, bench.job_throughput(1e9, 2, world, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        mx, gbs = out[r]
        assert mx == 150.0
        assert gbs == pytest.approx(2 * 1e9 * 2 / 0.150 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(2e9, 4, 1, 1000.0) == pytest.approx(8.0)
