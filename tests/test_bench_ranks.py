"""The multi-GPU path of bench.py is replicas only (every rank evaluates its own
states, no data-path collective).  Its host-side logic -- max over ranks of the
timed region, whole-job evals/s -- is checked here with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 200.0][rank]
    total, value = bench.aggregate_ranks(ms, 32 * 5, world, torch.device("cpu"))
    out[rank] = (total, value)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        total, value = out[r]
        assert total == pytest.approx(200.0)
        assert value == pytest.approx(2 * 32 * 5 / 0.2)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    total, value = bench.aggregate_ranks(50.0, 10, 1, None)
    assert total == 50.0 and value == pytest.approx(200.0)
