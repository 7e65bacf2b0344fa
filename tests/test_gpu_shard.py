"""Shards on the GPU: a global grid split over several contexts that exchange
faces every iteration through communication endpoints (the paper's
inter-process transport), bit for bit against the oracle's undecomposed
sweep -- all shards in one process, and two processes sharing one GPU
through CUDA IPC endpoints (only stream-level event waits cross the
processes; no kernel waits on another process)."""
import os
import socket

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def od():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_12734_gb300 import build
    build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


@pytest.mark.parametrize("path", ["per_chare", "fused", "persistent"])
@pytest.mark.parametrize("gdims,shards,split", [((40, 36, 33), (2, 1, 1), (2, 2, 2)),
                                                ((41, 30, 35), (2, 2, 2), (1, 2, 3)),
                                                ((301, 77), (2, 2), (2, 1))])
def test_in_process_shards(od, path, gdims, shards, split):
    from paper_2605_12734_gb300.shard import ShardedJacobi
    iters = 9
    with ShardedJacobi(gdims, shards, split, seed=3, init_mode=1, path=path) as sj:
        sj.step(4)
        sj.step(iters - 4)
        got = sj.read()
    want = oracle.solve(*gdims, 3, 1, iters) if len(gdims) == 3 else oracle.solve_2d(*gdims, 3, 1, iters)
    assert np.array_equal(bits(got), bits(want))


def test_shard_initial_field_and_faces(od):
    # a shard's initial field is the global field on its box, and an export of
    # a face is the global field's boundary layer there
    gdims, off, ext = (30, 20, 25), (10, 4, 7), (12, 9, 11)
    G = oracle.init_padded(*gdims, 8, 1)
    with od.Jacobi3D(*ext, split=(2, 1, 2), seed=8, init_mode=1, gdims=gdims, goff=off, path="fused") as s:
        u = s.read().reshape(ext[::-1])
        x0, y0, z0 = off
        nx, ny, nz = ext
        assert np.array_equal(bits(u), bits(G[z0 + 1:z0 + nz + 1, y0 + 1:y0 + ny + 1, x0 + 1:x0 + nx + 1]))
        f0 = np.empty(nz * ny)
        s.face_copy(0, 0, f0)     # x- boundary layer
        assert np.array_equal(bits(f0), bits(G[z0 + 1:z0 + nz + 1, y0 + 1:y0 + ny + 1, x0 + 1].ravel()))
        f5 = np.empty(ny * nx)
        s.face_copy(5, 0, f5)     # z+ boundary layer
        assert np.array_equal(bits(f5), bits(G[z0 + nz, y0 + 1:y0 + ny + 1, x0 + 1:x0 + nx + 1].ravel()))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, gdims, shards, split, iters, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2605_12734_gb300 as pkg
    from paper_2605_12734_gb300.shard import IpcTransport, ProcessShard, ShardPlan, _make_solver
    plan = ShardPlan(gdims, shards)
    stream = torch.cuda.Stream(device=0)
    solver = _make_solver(pkg, plan, rank, split, stream.cuda_stream, seed=4, init_mode=1, path="fused", device=0)
    tr = IpcTransport(plan, rank, 0, stream.cuda_stream)
    sh = ProcessShard(plan, rank, solver, tr)
    sh.step(iters)
    sh.drain()
    u = solver.read()
    out[rank] = (plan.origin(rank), plan.extents(rank), u)
    dist.barrier()  # every peer is done with this process's endpoint
    stream.synchronize()
    solver.close()
    tr.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("gdims,shards", [((48, 40, 36), (2, 1, 1)), ((96, 61), (2, 1))])
def test_two_processes_share_one_gpu_through_ipc(od, gdims, shards):
    import torch.multiprocessing as mp
    iters, world = 7, 2
    split = (2, 2, 2) if len(gdims) == 3 else (2, 2)
    with mp.get_context("spawn").Manager() as man:  # no fork after CUDA was initialised
        out = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), gdims, shards, split, iters, out), nprocs=world, join=True)
        res = dict(out)
    got = np.zeros(gdims[::-1])
    for r in range(world):
        o, e, u = res[r]
        got[tuple(slice(a, a + b) for a, b in zip(o, e))[::-1]] = u.reshape(e[::-1])
    want = oracle.solve(*gdims, 4, 1, iters) if len(gdims) == 3 else oracle.solve_2d(*gdims, 4, 1, iters)
    assert np.array_equal(bits(got.ravel()), bits(want))
