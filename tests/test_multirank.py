"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, each timing its
own replica, aggregate to the slowest rank's time and all ranks' cell updates
(replicas only: the method has no exchange step between GPUs)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 12.5][rank]
    e2e = [30.0, 20.0][rank]
    value, e2e_value, ms_max, e2e_max = bench.aggregate_ranks(ms, e2e, 1000, 4, world)
    out[rank] = (value, e2e_value, ms_max, e2e_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_to_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, e2e_value, ms_max, e2e_max = out[r]
        assert ms_max == 12.5 and e2e_max == 30.0
        assert value == pytest.approx(2 * 1000 * 4 / 12.5e-3 / 1e6)
        assert e2e_value == pytest.approx(2 * 1000 * 4 / 30e-3 / 1e6)


def test_single_rank_calls_no_collective():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    value, e2e_value, ms_max, _ = bench.aggregate_ranks(8.0, 16.0, 500, 2, 1)
    assert ms_max == 8.0 and value == pytest.approx(500 * 2 / 8e-3 / 1e6)
