"""The N > 1 bench path on CPU: replicas, gloo timing reduction (max over ranks), whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 1000.0 * (rank + 1)            # rank r pretends its K steps took (r + 1) s
    t_max = bench.max_over_ranks(t, dist)
    rate = bench.whole_job_rate(world, 3, t_max / 1e3)
    out[rank] = (t_max, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    import torch.multiprocessing as mp
    world = 2
    # spawned, not forked: this process may already run threads (the library's host pool)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t_max, rate = out[r]
        assert t_max == 2000.0               # the slowest rank sets the time
        assert abs(rate - 2 * 3 / 2.0) < 1e-12  # all ranks' units / slowest time


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(5.0) == 5.0
    assert bench.whole_job_rate(1, 2, 4.0) == 0.5
