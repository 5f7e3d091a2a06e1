"""Sharding one batch across GPUs, checked on one GPU: the batch split by sim_partition
into contiguous node-balanced ranges, each range stepped by its own handle, gives bit for
bit the state the unsharded handle gives (snakes are independent, and a snake's result
does not depend on the warp or queue position it gets).  The ranges run one after
another here; on several GPUs they run side by side with no exchange."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_02833_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _run(w, s, steps):
    from paper_1904_02833_gb300.sim import SnakeSim
    g = SnakeSim(w, s)
    g.step(steps, graph=True)
    st = g.state_host()
    st["lam"] = g.lam().cpu().numpy()
    g.close()
    return st


@pytest.mark.parametrize("parts,warm", [(2, 0), (3, 1)])
def test_sharded_batch_equals_unsharded_bit_for_bit(parts, warm):
    from paper_1904_02833_gb300.sim import partition
    w = W.learned(n=600, seed=4)
    s = W.solver_settings(iters=5000, tol=1e-4, warm=warm, beta=0.5)
    whole = _run(w, s, 3)
    first = partition(w, parts)
    nodes = np.concatenate([[0], np.cumsum(W.n_nodes(w))])
    links = np.concatenate([[0], np.cumsum(w["n_links"])])
    for p in range(parts):
        a, b = int(first[p]), int(first[p + 1])
        part = _run(W.subset(w, np.arange(a, b)), s, 3)
        na, nb, la, lb = int(nodes[a]), int(nodes[b]), int(links[a]), int(links[b])
        for k, sl in (("pos", slice(na, nb)), ("vel", slice(na, nb)), ("lam", slice(na, nb)),
                      ("press", slice(la, lb)), ("resid", slice(a, b)), ("iters", slice(a, b))):
            assert np.array_equal(part[k], whole[k][sl]), (p, k)
