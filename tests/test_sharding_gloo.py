"""The N > 1 path, run as two gloo ranks on CPU: each rank evaluates its own
points (here with the FP64 oracle), the ranks' shards partition the point set,
the per-rank results equal the single-process evaluation of the same points,
and the step time is reduced with MAX."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1605_01244_gb300 import sharding
from paper_1605_01244_gb300 import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = wl.gaussian_coeffs((8, 6, 10), 3.0, seed=0)
    x_all = wl.uniform_points(101, seed=1)
    a, b = sharding.shard_range(len(x_all), rank, world)
    f = oracle.forward(c, x_all[a:b])
    t = sharding.max_over_ranks(1.0 + rank)
    out[rank] = (a, b, f, t, sharding.point_seed(rank))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_points_and_reduce_time():
    import oracle
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    res = [out[r] for r in range(world)]
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == 101
    assert all(r[3] == 2.0 for r in res)                      # MAX over ranks
    assert res[0][4] != res[1][4]                              # distinct batch seeds
    c = wl.gaussian_coeffs((8, 6, 10), 3.0, seed=0)
    full = oracle.forward(c, wl.uniform_points(101, seed=1))
    got = np.concatenate([res[0][2], res[1][2]])
    assert np.array_equal(got, full)


def test_shard_ranges_cover_exactly():
    for M in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            spans = [sharding.shard_range(M, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == M
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
