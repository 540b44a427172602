"""The N > 1 path of the benchmark (independent replicas, one per GPU) on
CPU: two gloo ranks aggregate their timings the way bench.py does -- the
slowest rank's time and the units of every rank."""
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

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (100 + 50 r) ms for 1e12 (r + 1) units
    ms, value = bench.aggregate(100.0 + 50.0 * rank, 1e12 * (rank + 1), world)
    out[rank] = (ms, value, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        ms, value, env = out[r]
        assert ms == 150.0                       # max over ranks
        assert value == pytest.approx(3e12 / 0.150)  # all ranks' units / max time
        assert env == (r, world, r)


def test_single_process_aggregation():
    import bench
    ms, value = bench.aggregate(200.0, 4e12, 1)
    assert ms == 200.0 and value == pytest.approx(2e13)
