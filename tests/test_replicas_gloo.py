"""The N > 1 benchmark path: independent replicas, max-over-ranks timing.

Runs two gloo ranks on the CPU (no GPU, no collective on the data path):
each rank reports its own time, the job time is the slowest rank's and the
throughput counts the steps of every replica.
"""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 * (rank + 1)          # rank 1 is the slower replica
    value, ms = bench.replica_throughput(ms_local, steps=50, dist=dist, device="cpu")
    dist.barrier()
    out.put((rank, value, ms))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 50 / 0.2)
