"""The multi-GPU path of bench.py is replicas only: every rank advances its own
copy of the workload, ranks meet at a barrier, the job time is the slowest
rank's and the job rate counts all ranks' points.  Checked here with two gloo
ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = 10.0 * (rank + 1)                 # the ranks' own timed regions differ
    job_ms = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (job_ms, bench.job_rate(world, 64 ** 3, 5, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_slowest_rank_and_sum_points():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] == pytest.approx(2 * 64 ** 3 * 5 / 0.020)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 100, 4, 2.0) == pytest.approx(200000.0)
