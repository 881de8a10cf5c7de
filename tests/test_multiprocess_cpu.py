"""The N-GPU path of the benchmark is N independent replicas (one frame per rank, weak
scaling, no collective on the data path); its only cross-rank step is the timing
aggregation, tested here with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    my_ms = [100.0, 250.0][rank]                 # rank 1 is the slow one
    job_ms, value = bench.aggregate(my_ms, 1000, dist, torch.device("cpu"))
    dist.barrier()
    out.put((rank, job_ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for rank, job_ms, value in res:
        assert job_ms == 250.0                      # max over ranks
        assert value == pytest.approx(2 * 1000 / 0.25)   # units of all ranks over the job time


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(50.0, 10) == (50.0, 200.0)
