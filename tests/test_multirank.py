"""The N > 1 path of bench.py on CPU: world-size-2 gloo process group. Ranks
render disjoint shares of the orbit views (replicas over views), and the job's
time is the slowest rank's while its samples are the sum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    views = bench.shard_views(rank, world, 8, 12)
    ms = 10.0 + rank  # rank 1 is the slowest
    e2e = 1.0 + 2 * rank
    samples = 100.0 * (rank + 1)
    out = bench.reduce_job(ms, e2e, samples, world, device="cpu")
    q.put((rank, views, out))
    dist.destroy_process_group()


def test_views_sharded_and_job_reduced_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, views, out = q.get(timeout=120)
        res[r] = (views, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    v0, v1 = res[0][0], res[1][0]
    assert v0[:4] == [0, 2, 4, 6] and v1[:4] == [1, 3, 5, 7]
    assert not set(v0[:4]) & set(v1[:4])  # each frame of a round is rendered once
    for r in (0, 1):
        assert res[r][1] == (11.0, 3.0, 300.0)


def test_single_rank_is_identity():
    import bench
    assert bench.shard_views(0, 1, 8, 10) == [0, 1, 2, 3, 4, 5, 6, 7, 0, 1]
    assert bench.reduce_job(5.0, 2.0, 7.0, 1) == (5.0, 2.0, 7.0)
