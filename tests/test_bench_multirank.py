"""The replica (N > 1) aggregation of bench.py on CPU with gloo, world size 2:
each rank renders its own face, the job's step time is the slowest rank's
and its throughput counts the samples of every rank."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, v = bench.aggregate(10.0 + 5.0 * rank, 1_048_576, world, None)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_replica_aggregation_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 15.0                                   # max over ranks
        assert abs(v - 2 * 1_048_576 / 0.015 / 1e6) < 1e-9  # all ranks' samples / slowest time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate(20.0, 1_000_000, 1) == (20.0, 50.0)
