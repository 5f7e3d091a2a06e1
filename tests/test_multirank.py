"""Multi-GPU host logic on the CPU (gloo, world size 2): one seeded batch is split into
contiguous snake ranges balanced by node count (sim_partition, a host call of the
library), each rank simulates its own range with no data-path collective, and the
whole-job throughput is the units of all ranks over the slowest rank's time."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W


def _loads(w, first):
    pre = np.concatenate([[0], np.cumsum(W.n_nodes(w))])
    return pre[first[1:]] - pre[first[:-1]]


@pytest.mark.parametrize("parts", [1, 2, 3, 4, 7, 8])
def test_partition_covers_the_batch_in_node_balanced_ranges(parts):
    from paper_1904_02833_gb300.sim import partition
    w = W.learned(n=3000, seed=4)
    first = partition(w, parts)
    assert first[0] == 0 and first[-1] == 3000 and (np.diff(first) >= 0).all()
    loads = _loads(w, first)
    ideal = W.n_nodes(w).sum() / parts
    # every part within one snake's nodes of the ideal share
    assert np.abs(loads - ideal).max() <= W.n_nodes(w).max()


def test_partition_edge_cases():
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.sim import partition, make_params
    w = W.learned(n=5, seed=9)
    # more parts than snakes: some ranges are empty, still a cover
    first = partition(w, 9)
    assert first[0] == 0 and first[-1] == 5 and (np.diff(first) >= 0).all()
    assert (np.diff(first) <= 1).all()
    # equal snakes split evenly
    e = W.learned(n=12, seed=9)
    e["n_links"][:] = 3
    assert list(partition(e, 4)) == [0, 3, 6, 9, 12]
    # a ragged batch whose largest snake holds over half the nodes
    r = W.learned(n=4, seed=9)
    r["n_links"][:] = [1, 8, 1, 1]
    f = partition(r, 2)
    assert list(f) in ([0, 1, 4], [0, 2, 4])
    lib = N.load()
    p = make_params(w)
    out = np.zeros(3, np.int32)
    assert lib.sim_partition(5, p, 0, out.ctypes.data_as(N.P)) == N.SIM_EINVAL
    assert lib.sim_partition(0, p, 2, out.ctypes.data_as(N.P)) == N.SIM_EINVAL


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.N_SNAKES = 500
    w_all = bench.eval_batch(world)
    w = bench.shard(w_all, rank, world)
    # the first snake's parameters identify the range (yaw drawn per snake)
    t_local = 2.0 if rank == 0 else 3.0
    n_local = len(w["n_links"])
    value, t_max, units = bench.aggregate(t_local, n_local * 5, dist)
    out[rank] = (n_local, int(W.n_nodes(w).sum()), float(w["yaw0"][0]), float(w["yaw0"][-1]),
                 value, t_max, units, float(w_all["yaw0"][0]), float(w_all["yaw0"][-1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_one_batch_and_aggregate():
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
    (n0, m0, a0, b0, v0, t0, u0, f0, l0), (n1, m1, a1, b1, v1, t1, u1, f1, l1) = out[0], out[1]
    assert n0 + n1 == 1000                        # the two ranges cover the batch
    assert a0 == f0 and b1 == l1                  # rank 0 starts it, rank 1 ends it
    assert abs(m0 - m1) <= 81                     # node counts within one snake
    assert t0 == t1 == 3.0                        # slowest rank's time
    assert u0 == u1 == 5.0 * 1000                 # all ranks' env-steps
    assert v0 == v1 == pytest.approx(5000.0 / 3.0)


def test_single_process_aggregation_without_a_process_group():
    import bench
    value, t, u = bench.aggregate(2.0, 100, None)
    assert value == 50.0 and t == 2.0 and u == 100.0
