"""The benchmark's multi-GPU path runs one independent replica per rank
(the solve has no exchange between GPUs) and reports the slowest rank's time
and the updates of all ranks.  This checks that combination with two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 55.0][rank]          # rank 1 is the slowest
    updates = [1.0e9, 1.0e9][rank]   # same replica on every rank
    t, value = bench.combine_ranks(ms, updates, world, "cpu")
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_combination():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, value = res[rank]
        assert t == 55.0
        assert value == pytest.approx(2.0e9 / 0.055)


def test_single_rank_needs_no_group():
    import bench
    t, value = bench.combine_ranks(20.0, 1e9, 1, "cpu")
    assert t == 20.0 and value == pytest.approx(5e10)
