"""The N > 1 path of bench.py on the CPU: world size 2 over gloo.

Ranks are independent replicas (the solves of different problems share no
data), so the only cross-rank steps are a barrier and the max-over-ranks job
time from which whole-job throughput is computed."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    # rank r pretends its 4 solves took (r + 1) seconds
    value, t = bench.aggregate(dist, world, 4, float(rank + 1))
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_replicas_aggregate_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == 2.0                      # slowest rank's time
        assert value == pytest.approx(world * 4 / 2.0)
