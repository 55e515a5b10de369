"""The N > 1 path of bench.py (independent replicas, one per rank): the job time is the maximum
over ranks and the value counts every rank's units.  world_size 2 on CPU with the gloo backend."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    value, t = bench.replica_throughput(1.0 + rank, 1000.0, world, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_throughput_world2():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(2):
        value, t = out[r]
        assert t == 2.0                 # max over ranks
        assert value == 2 * 1000.0 / 2.0  # all ranks' units / job time


def test_single_rank():
    import bench

    assert bench.replica_throughput(0.5, 10.0, 1) == (20.0, 0.5)
