"""The benchmark's multi-rank plumbing on CPU: two gloo ranks (replicas)
aggregate whole-job bytes (sum) and time (max over ranks), as the N-GPU bench
does with NCCL; the virtual-rank path itself has no data-path collective."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r = bench.dist_init("gloo")
    assert (w, r) == (world, rank)
    bench.barrier()
    b, t = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank)
    out[rank] = (b, t)
    bench.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        for r in range(world):
            assert out[r] == (3000.0, 1.5)


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)
