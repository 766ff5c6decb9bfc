"""The N > 1 path with two gloo ranks.  CPU: each rank evaluates its own
points with the FP64 oracle, the ranks' shards partition the point set, the
per-rank results equal the single-process evaluation of the same points, and
the step time is reduced with MAX.  GPU: the same through the library's plans
and its timed sharded step (sharding.timed_steps), both ranks on one device."""
import os
import socket

import numpy as np
import pytest
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


# ---- GPU: the library's sharded step, two ranks ------------------------------
# Both ranks run on cuda:0 as separate processes.  Their kernels are
# independent (no kernel waits on another rank); the only exchanges are gloo
# collectives on the host.

def _lib_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_1605_01244_gb300 import sharding as sh
    from paper_1605_01244_gb300.nfft import Plan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cuda", 0)
    c = torch.from_numpy(wl.gaussian_coeffs((32, 32, 32), 6.0, seed=0)).to(dev)
    x_all = wl.mixed_points(20001, 0.02, seed=1)
    a, b = sh.shard_range(len(x_all), rank, world)
    x = torch.from_numpy(x_all[a:b]).to(dev)
    plan = Plan((32, 32, 32), b - a, m=6, precision="f64")
    f = torch.empty(b - a, dtype=torch.complex128, device=dev)

    def step():
        plan.set_points(x)
        plan.eval(c, out=f)

    step()
    ms = sh.timed_steps(step, 3, torch.cuda.current_stream(dev), dev)
    own = sh.max_over_ranks(1.0 + rank, dev)
    parts = [None] * world
    dist.all_gather_object(parts, f.cpu().numpy())
    plan.close()
    out[rank] = (ms, own, np.concatenate(parts))
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_ranks_through_the_library_on_one_gpu():
    import torch
    import oracle
    from paper_1605_01244_gb300 import build
    from paper_1605_01244_gb300.nfft import Plan
    build.build()
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_lib_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    res = [out[r] for r in range(world)]
    assert res[0][0] == res[1][0] > 0            # the step time reduced with MAX on both ranks
    assert res[0][1] == res[1][1] == 2.0
    assert np.array_equal(res[0][2], res[1][2])  # both ranks gathered the same result
    # against one process evaluating all points, and against the direct sum
    c_np = wl.gaussian_coeffs((32, 32, 32), 6.0, seed=0)
    x_all = wl.mixed_points(20001, 0.02, seed=1)
    plan = Plan((32, 32, 32), len(x_all), m=6, precision="f64")
    plan.set_points(torch.from_numpy(x_all).cuda())
    one = plan.eval(torch.from_numpy(c_np).cuda()).cpu().numpy()
    plan.close()
    got = res[0][2]
    assert np.max(np.abs(got - one)) <= 1e-14 * np.max(np.abs(one))
    idx = np.random.default_rng(5).choice(len(x_all), 1500, replace=False)
    fd = oracle.forward(c_np, x_all[idx])
    assert np.linalg.norm(got[idx] - fd) / np.linalg.norm(fd) <= 1e-12
