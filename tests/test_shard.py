"""One mesh on several ranks by source partition (paper_1606_00247_gb300/shard.py):
the partition covers every tet once in compact Morton ranges, and the sum of
the shards' potentials equals the whole mesh's -- with two gloo ranks on CPU
(the oracle's direct sum evaluates each shard) and, on the GPU, with the
library evaluating each shard's own plan."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1606_00247_gb300 import inputs
from paper_1606_00247_gb300.shard import morton_partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_tet_once():
    nodes, tets = inputs.unit_cube(6)
    for r in (1, 2, 3, 8):
        parts = morton_partition(nodes, tets, r)
        assert len(parts) == r
        allt = np.concatenate(parts)
        assert np.array_equal(np.sort(allt), np.arange(len(tets)))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    # two halves of a Kuhn cube by Morton order: each half is one compact block of cells
    a, b = morton_partition(nodes, tets, 2)
    ca = nodes[tets[a]].mean(axis=1)
    cb = nodes[tets[b]].mean(axis=1)
    assert np.any([ca[:, k].max() <= cb[:, k].min() + 1e-12 for k in range(3)])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    from paper_1606_00247_gb300 import inputs
    from paper_1606_00247_gb300.shard import allreduce_u, morton_partition

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nodes, tets = inputs.unit_cube(4)
    M = inputs.gaussian_unit_m(nodes.shape[0], seed=31)
    mine = morton_partition(nodes, tets, world)[rank]
    u = torch.as_tensor(oracle.direct(nodes, tets[mine], M, nthreads=1))
    allreduce_u(u)
    out[rank] = u.numpy()
    dist.destroy_process_group()


def test_two_rank_source_partition_sums_to_the_whole_mesh(orc):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    nodes, tets = inputs.unit_cube(4)
    M = inputs.gaussian_unit_m(nodes.shape[0], seed=31)
    ref = orc.direct(nodes, tets, M)
    for r in range(2):
        assert np.abs(out[r] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.gpu
def test_gpu_shards_sum_to_the_whole_mesh():
    """Each shard is a plan of its own tets over all nodes (FP64, p = 8): the
    sum of the shards' u equals the whole mesh's u within the FMM truncation
    of the two different trees."""
    from paper_1606_00247_gb300.api import Plan

    nodes, tets = inputs.sphere(h=0.12)
    M = torch.as_tensor(inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=33), device="cuda")
    u_full, _ = Plan(nodes, tets, p=8, leaf_size=32, theta=0.5, near_mode=1, max_batch=2).eval(M)
    u_sum = torch.zeros_like(u_full)
    for part in morton_partition(nodes, tets, 3):
        u_k, _ = Plan(nodes, tets[part], p=8, leaf_size=32, theta=0.5, near_mode=1, max_batch=2).eval(M)
        u_sum += u_k
    err = float(torch.linalg.norm(u_sum - u_full) / torch.linalg.norm(u_full))
    assert err < 1e-5, err
