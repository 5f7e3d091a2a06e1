"""Multi-rank logic of the benchmark on CPU (gloo, world size 2): every rank simulates its
own shard of snakes (no data-path collective); the whole-job throughput is the units of
all ranks over the slowest rank's time."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    # shards differ per rank and stay disjoint from the training seeds
    seed = bench.shard_seed(rank)
    assert seed < W.training_seeds(1)[0]
    w = W.learned(n=16, seed=seed)
    t_local = 2.0 if rank == 0 else 3.0
    value, t_max, units = bench.aggregate(t_local, 16 * 5, dist)
    out[rank] = (seed, float(w["yaw0"][0]), value, t_max, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_and_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (s0, y0, v0, t0, u0), (s1, y1, v1, t1, u1) = out[0], out[1]
    assert s0 != s1 and y0 != y1          # different snakes on each rank
    assert t0 == t1 == 3.0                # slowest rank's time
    assert u0 == u1 == 160.0              # all ranks' env-steps
    assert v0 == v1 == pytest.approx(160.0 / 3.0)


def test_single_process_aggregation_without_a_process_group():
    import bench
    value, t, u = bench.aggregate(2.0, 100, None)
    assert value == 50.0 and t == 2.0 and u == 100.0
