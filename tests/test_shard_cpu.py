"""Shards on the CPU: the split of a global grid into shards, and the
inter-process face-exchange protocol (copy into the sender's buffer, control
message with offset and event index, copy into the receiver's ghost layer,
acknowledgement before a region is reused) run by gloo ranks.  Each rank's
local solver here is the oracle's sweep of its padded sub-box and the
transport stages faces on the host; the result must equal the oracle's
undecomposed sweep bit for bit."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2605_12734_gb300.shard import OPPOSITE, ShardPlan, split_edges

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("gdims,shards", [((10, 7, 9), (2, 1, 1)), ((10, 7, 9), (2, 3, 2)), ((5, 6), (2, 3)),
                                          ((3, 3, 3), (3, 3, 3))])
def test_plan_tiles_the_grid(gdims, shards):
    P = ShardPlan(gdims, shards)
    assert P.n == int(np.prod(shards))
    cover = np.zeros(gdims[::-1], dtype=np.int32)
    for r in range(P.n):
        o, e = P.origin(r), P.extents(r)
        cover[tuple(slice(a, a + b) for a, b in zip(o, e))[::-1]] += 1
        for f in range(P.nfaces):
            q = P.nbr[r][f]
            if q < 0:  # a domain face
                a = f // 2
                assert (o[a] == 0) if f % 2 == 0 else (o[a] + e[a] == gdims[a])
                continue
            assert P.nbr[q][OPPOSITE[f]] == r
            assert P.face_cells(r, f) == P.face_cells(q, OPPOSITE[f])
        # the two regions of every linked face are disjoint and inside the buffer
        spans = sorted((a, a + P.face_cells(r, f)) for f, regs in P.offset[r].items() for a in regs)
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0
        assert not spans or spans[-1][1] <= P.doubles[r]
    assert (cover == 1).all()


def test_split_edges_matches_oracle():
    for n, p in [(10, 3), (512, 16), (7, 7), (100, 6)]:
        assert split_edges(n, p) == list(oracle.split(n, p))


class OracleShard:
    """A shard's local solver on the CPU: its padded sub-box of the global
    initial field, swept by the oracle with its ghost layers held fixed."""

    def __init__(self, plan, r, seed, mode):
        if plan.dim == 3:
            G = oracle.init_padded(*plan.gdims, seed, mode)
        else:
            G = oracle.init_padded_2d(*plan.gdims, seed, mode)
        sl = tuple(slice(o, o + e + 2) for o, e in zip(plan.origin(r), plan.extents(r)))[::-1]
        self.P = np.ascontiguousarray(G[sl])
        self.dim = plan.dim

    def step(self, n):
        self.P = oracle.sweep(self.P, n) if self.dim == 3 else oracle.sweep_2d(self.P, n)

    def _layer(self, f, ghost):
        a, hi = f // 2, f % 2
        n = self.P.shape[::-1][a] - 2            # interior extent along axis a
        i = (n + 1 if hi else 0) if ghost else (n if hi else 1)
        idx = [slice(1, -1)] * self.dim
        idx[a] = i
        return tuple(idx[::-1])

    def face_copy(self, f, direction, buf):
        lay = self._layer(f, ghost=direction == 1)
        if direction == 0:
            buf[:] = self.P[lay].ravel()
        else:
            self.P[lay] = np.asarray(buf).reshape(self.P[lay].shape)

    def interior(self):
        return self.P[tuple([slice(1, -1)] * self.dim)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, gdims, shards, iters, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2605_12734_gb300.shard import HostTransport, ProcessShard, ShardPlan
    plan = ShardPlan(gdims, shards)
    solver = OracleShard(plan, rank, seed=5, mode=1)
    sh = ProcessShard(plan, rank, solver, HostTransport(plan, rank))
    sh.step(iters // 2)
    sh.step(iters - iters // 2)
    sh.drain()
    out[rank] = (plan.origin(rank), plan.extents(rank), solver.interior().copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("gdims,shards,iters", [((12, 9, 10), (2, 1, 1), 7), ((12, 9, 10), (2, 1, 2), 5),
                                                 ((13, 8), (2, 2), 6)])
def test_process_shards_match_the_undecomposed_sweep(gdims, shards, iters):
    import torch.multiprocessing as mp
    world = int(np.prod(shards))
    with mp.get_context("spawn").Manager() as man:  # no fork after CUDA was initialised
        out = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), gdims, shards, iters, out), nprocs=world, join=True)
        res = dict(out)
    got = np.zeros(gdims[::-1])
    for r in range(world):
        o, e, u = res[r]
        got[tuple(slice(a, a + b) for a, b in zip(o, e))[::-1]] = u
    if len(gdims) == 3:
        want = oracle.solve(*gdims, 5, 1, iters)
    else:
        want = oracle.solve_2d(*gdims, 5, 1, iters)
    assert np.array_equal(got.ravel().view(np.uint64), want.view(np.uint64))
