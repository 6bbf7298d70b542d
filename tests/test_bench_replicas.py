"""Multi-GPU layout of the benchmark: replicas only (the slab solve is not sharded; every
rank marches its own copy).  The whole-job rate is the units of all ranks over the slowest
rank's time; checked here with two gloo ranks on the CPU."""
import os

import pytest

torch = pytest.importorskip("torch")


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, t_job = bench.whole_job_rate(1000.0, 1.0 + rank, world)  # rank 1 is the slow one
    out[rank] = (value, t_job)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        value, t_job = out[r]
        assert t_job == 2.0
        assert value == 2 * 1000.0 / 2.0


def test_single_rank_rate():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.whole_job_rate(500.0, 2.0, 1) == (250.0, 2.0)
