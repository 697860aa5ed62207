"""The multi-process bench path on CPU: world_size 2 over gloo, each rank with
its own work, no data-path collective; the value is all ranks' units over the
slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 100.0 * (rank + 1)  # rank 1 is the slowest
    bench.barrier(dist)
    value, ms_max = bench.aggregate(dist, 5, ms)
    out[rank] = (value, ms_max)
    dist.destroy_process_group()


def test_two_rank_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(world):
        value, ms_max = out[r]
        assert ms_max == pytest.approx(200.0)
        assert value == pytest.approx(2 * 5 / 0.2)
