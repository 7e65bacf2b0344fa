"""Shards: one global Jacobi grid split over several contexts -- the paper's
processes -- that exchange boundary faces every iteration through the
intra-node, inter-process transport (Sec. IV, transport item 2).

Each shard is a libod context holding a sub-box of the global grid
(``od_config.gnx`` ...), itself overdecomposed into chares.  Faces between
shards move as the paper describes: the sender copies its boundary layer
into its own pre-allocated communication buffer (``od_face_copy`` export,
copy 1) and records an event of its endpoint; a control message with the
buffer offset and the event index reaches the receiver, whose stream waits
on that event and copies from the sender's buffer into its ghost layer
(``od_face_copy`` import, copy 2); the receiver then records an
acknowledgement event so the sender may reuse the region two iterations
later (each outgoing face has two regions, alternating by iteration).

* ``ShardPlan``   the split of the global grid, neighbours, buffer offsets
                  and event indices (host logic only).
* ``ShardedJacobi`` every shard in this process (contexts on one GPU, local
                  endpoints, no control messages needed).
* ``ProcessShard`` this process's shard; peers are other processes (one
                  shard each, rank r = shard r) reached through their mapped
                  endpoints, control messages through ``torch.distributed``.
                  The solver and transport are parameters, so the protocol
                  also runs with host staging (``HostTransport``).
"""
from __future__ import annotations

import numpy as np

OPPOSITE = (1, 0, 3, 2, 5, 4)
CTRL_TAG, ACK_TAG = 100, 200


def split_edges(n: int, p: int) -> list[int]:
    """Balanced block edges: the first n mod p blocks get one more cell."""
    if p < 1 or p > n:
        raise ValueError(f"cannot split {n} cells into {p} blocks")
    q, r = divmod(n, p)
    e = [0]
    for i in range(p):
        e.append(e[-1] + q + (1 if i < r else 0))
    return e


class ShardPlan:
    """Split of a global grid into shards (x fastest: rank = ix + sx*(iy + sy*iz)).

    3D: gdims = (gnx, gny, gnz), shards = (sx, sy, sz), faces 0..5.
    2D: gdims = (gnx, gny), shards = (sx, sy), faces 0..3 (x-, x+, y-, y+).
    For every shard and face with a neighbour shard the sender's buffer holds
    two regions (by iteration parity); event 2f+s signals region s of face f
    filled, event 2F+2f+s acknowledges an import into face f from region s
    (F = number of faces)."""

    def __init__(self, gdims, shards):
        self.dim = len(gdims)
        if self.dim not in (2, 3) or len(shards) != self.dim:
            raise ValueError("gdims and shards must both have 2 or 3 entries")
        self.gdims = tuple(int(v) for v in gdims)
        self.shards = tuple(int(v) for v in shards)
        self.nfaces = 2 * self.dim
        self.edges = [split_edges(n, p) for n, p in zip(self.gdims, self.shards)]
        self.n = int(np.prod(self.shards))
        self.boxes, self.nbr = [], []
        for r in range(self.n):
            idx, rem = [], r
            for p in self.shards:
                idx.append(rem % p)
                rem //= p
            box = []
            for a in range(self.dim):
                e = self.edges[a]
                box += [e[idx[a]], e[idx[a] + 1] - e[idx[a]]]
            self.boxes.append(tuple(box))
            nb, stride = [], 1
            for a in range(self.dim):
                nb.append(r - stride if idx[a] > 0 else -1)
                nb.append(r + stride if idx[a] < self.shards[a] - 1 else -1)
                stride *= self.shards[a]
            self.nbr.append(tuple(nb))
        # buffer layout: every face with a neighbour, two regions each
        self.offset, self.doubles = [], []
        for r in range(self.n):
            off, at = {}, 0
            for f in range(self.nfaces):
                if self.nbr[r][f] >= 0:
                    n = self.face_cells(r, f)
                    off[f] = (at, at + n)
                    at += 2 * n
            self.offset.append(off)
            self.doubles.append(max(at, 1))
        self.nevents = 4 * self.nfaces

    def extents(self, r):
        b = self.boxes[r]
        return tuple(b[2 * a + 1] for a in range(self.dim))

    def origin(self, r):
        b = self.boxes[r]
        return tuple(b[2 * a] for a in range(self.dim))

    def face_cells(self, r, f) -> int:
        ext = self.extents(r)
        return int(np.prod([e for a, e in enumerate(ext) if a != f // 2]))

    def data_event(self, f, slot):
        return 2 * f + slot

    def ack_event(self, f, slot):
        return 2 * self.nfaces + 2 * f + slot

    def linked_faces(self, r):
        return [f for f in range(self.nfaces) if self.nbr[r][f] >= 0]


def _make_solver(pkg, plan, r, split, stream, **kw):
    ext, org = plan.extents(r), plan.origin(r)
    if plan.dim == 2:
        return pkg.Jacobi2D(ext[0], ext[1], split=split, gdims=plan.gdims, goff=org, stream=stream, **kw)
    return pkg.Jacobi3D(*ext, split=split, gdims=plan.gdims, goff=org, stream=stream, **kw)


class ShardedJacobi:
    """Every shard of `plan` in this process, one context and one stream each,
    on one GPU.  split: chares per shard (per axis)."""

    def __init__(self, gdims, shards, split, *, device: int = 0, **kw):
        import torch
        import paper_2605_12734_gb300 as pkg
        self.plan = ShardPlan(gdims, shards)
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(self.plan.n)]
        self.solvers = [_make_solver(pkg, self.plan, r, split, self.streams[r].cuda_stream, device=device, **kw)
                        for r in range(self.plan.n)]
        self.comms = [pkg.Comm.create(8 * self.plan.doubles[r], self.plan.nevents, device)
                      for r in range(self.plan.n)]
        self.t = 0

    def step(self, iters: int) -> None:
        P = self.plan
        for _ in range(int(iters)):
            t, slot = self.t, self.t & 1
            for s in self.solvers:
                s.step(1)
            for r in range(P.n):  # copy 1: boundary layer -> own buffer, then signal
                st = self.streams[r].cuda_stream
                for f in P.linked_faces(r):
                    q = P.nbr[r][f]
                    if t >= 2:  # the receiver has finished with this region (iteration t-2)
                        self.comms[q].wait(P.ack_event(OPPOSITE[f], slot), st)
                    self.solvers[r].face_copy(f, 0, self.comms[r].ptr + 8 * P.offset[r][f][slot])
                    self.comms[r].record(P.data_event(f, slot), st)
            for q in range(P.n):  # copy 2: sender's buffer -> ghost layer, then acknowledge
                st = self.streams[q].cuda_stream
                for g in P.linked_faces(q):
                    r, f = P.nbr[q][g], OPPOSITE[g]
                    self.comms[r].wait(P.data_event(f, slot), st)
                    self.solvers[q].face_copy(g, 1, self.comms[r].ptr + 8 * P.offset[r][f][slot])
                    self.comms[q].record(P.ack_event(g, slot), st)
            self.t += 1

    def read(self) -> np.ndarray:
        """The global interior, x fastest."""
        out = np.empty(int(np.prod(self.plan.gdims)), dtype=np.float64)
        g = out.reshape(self.plan.gdims[::-1])
        for r, s in enumerate(self.solvers):
            u = s.read().reshape(self.plan.extents(r)[::-1])
            sl = tuple(slice(o, o + e) for o, e in zip(self.plan.origin(r), self.plan.extents(r)))[::-1]
            g[sl] = u
        return out

    def close(self) -> None:
        for s in self.streams:
            s.synchronize()
        for s in self.solvers:
            s.close()
        for c in self.comms:
            c.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------ one shard per process

class IpcTransport:
    """Peer endpoints mapped through CUDA IPC; control messages carry the
    offset and the event index (no payload)."""

    def __init__(self, plan, rank, device, stream):
        import torch.distributed as dist
        import paper_2605_12734_gb300 as pkg
        self.plan, self.rank, self.stream = plan, rank, stream
        self.own = pkg.Comm.create(8 * plan.doubles[rank], plan.nevents, device)
        blobs = [None] * plan.n
        dist.all_gather_object(blobs, self.own.handles())
        self.peer = {q: pkg.Comm.open(blobs[q], device) for q in set(plan.nbr[rank]) if q >= 0}

    def region(self, f, slot):
        return self.own.ptr + 8 * self.plan.offset[self.rank][f][slot]

    def after_export(self, f, slot):
        self.own.record(self.plan.data_event(f, slot), self.stream)
        return [self.plan.offset[self.rank][f][slot], self.plan.data_event(f, slot)]

    def before_import(self, r, msg):
        off, ev = msg
        self.peer[r].wait(ev, self.stream)
        return self.peer[r].ptr + 8 * off

    def after_import(self, g, slot):
        self.own.record(self.plan.ack_event(g, slot), self.stream)

    def before_reuse(self, q, f, slot):
        self.peer[q].wait(self.plan.ack_event(OPPOSITE[f], slot), self.stream)

    def payload(self, f, slot):
        return None

    def close(self):
        for c in self.peer.values():
            c.close()
        self.own.close()


class HostTransport:
    """Host staging (CPU ranks): each region is a host array and the control
    message carries the face itself."""

    def __init__(self, plan, rank):
        self.plan, self.rank = plan, rank
        self.buf = np.zeros(plan.doubles[rank], dtype=np.float64)
        self.inbox = {}

    def region(self, f, slot):
        a, n = self.plan.offset[self.rank][f][slot], self.plan.face_cells(self.rank, f)
        return self.buf[a:a + n]

    def after_export(self, f, slot):
        return [self.plan.offset[self.rank][f][slot], self.plan.data_event(f, slot)]

    def payload(self, f, slot):
        return self.region(f, slot)

    def before_import(self, r, msg, data=None):
        return data

    def after_import(self, g, slot):
        pass

    def before_reuse(self, q, f, slot):
        pass

    def close(self):
        pass


class ProcessShard:
    """Shard `rank` of `plan`, the others held by peer processes (torch.distributed
    initialised, world size = plan.n).  solver: a context-like object with
    step(1) and face_copy(face, dir, buf); transport: IpcTransport or
    HostTransport.  Every iteration: step, export and signal each linked
    face (after the receiver acknowledged the region's previous use), then
    receive, import and acknowledge each incoming face."""

    def __init__(self, plan: ShardPlan, rank: int, solver, transport):
        self.plan, self.rank, self.solver, self.tr = plan, rank, solver, transport
        self.t = 0
        # acknowledgements in flight: a send completes only once the peer has
        # posted the matching receive, which it does two iterations later
        self.acks = []

    def step(self, iters: int) -> None:
        import torch
        import torch.distributed as dist
        P, me = self.plan, self.rank
        faces = P.linked_faces(me)
        for _ in range(int(iters)):
            t, slot = self.t, self.t & 1
            self.solver.step(1)
            sends = []
            for f in faces:
                q = P.nbr[me][f]
                if t >= 2:  # region `slot` of face f was last read by q at iteration t-2
                    ack = torch.zeros(3, dtype=torch.int64)
                    dist.recv(ack, src=q, tag=ACK_TAG + OPPOSITE[f])
                    if int(ack[0]) != t - 2:
                        raise RuntimeError(f"shard {me}: acknowledgement for iteration {int(ack[0])}, "
                                           f"expected {t - 2}")
                    self.tr.before_reuse(q, f, slot)
                self.solver.face_copy(f, 0, self.tr.region(f, slot))
                ctrl = torch.tensor([t, f] + self.tr.after_export(f, slot), dtype=torch.int64)
                sends.append((ctrl, dist.isend(ctrl, dst=q, tag=CTRL_TAG + f)))
                data = self.tr.payload(f, slot)
                if data is not None:
                    td = torch.from_numpy(np.ascontiguousarray(data))
                    sends.append((td, dist.isend(td, dst=q, tag=CTRL_TAG + 10 + f)))
            for g in faces:
                r = P.nbr[me][g]
                ctrl = torch.zeros(4, dtype=torch.int64)
                dist.recv(ctrl, src=r, tag=CTRL_TAG + OPPOSITE[g])
                if int(ctrl[0]) != t or int(ctrl[1]) != OPPOSITE[g]:
                    raise RuntimeError(f"shard {me}: control message {ctrl.tolist()} out of order")
                msg = [int(ctrl[2]), int(ctrl[3])]
                if isinstance(self.tr, HostTransport):
                    data = torch.empty(P.face_cells(me, g), dtype=torch.float64)
                    dist.recv(data, src=r, tag=CTRL_TAG + 10 + OPPOSITE[g])
                    src = self.tr.before_import(r, msg, data.numpy())
                else:
                    src = self.tr.before_import(r, msg)
                self.solver.face_copy(g, 1, src)
                self.tr.after_import(g, slot)
                ack = torch.tensor([t, g, P.ack_event(g, slot)], dtype=torch.int64)
                self.acks.append((t, ack, dist.isend(ack, dst=r, tag=ACK_TAG + g)))
            # the peers have taken this iteration's control messages (they
            # answered with their own) and the acknowledgements of t-2
            for _, req in sends:
                req.wait()
            while self.acks and self.acks[0][0] <= t - 2:
                self.acks.pop(0)[2].wait()
            self.t += 1

    def drain(self) -> None:
        """Consume the acknowledgements of the last two iterations (so every
        message is matched before the process group goes away)."""
        import torch
        import torch.distributed as dist
        P, me = self.plan, self.rank
        for t in range(max(0, self.t - 2), self.t):
            for f in P.linked_faces(me):
                ack = torch.zeros(3, dtype=torch.int64)
                dist.recv(ack, src=P.nbr[me][f], tag=ACK_TAG + OPPOSITE[f])
        while self.acks:
            self.acks.pop(0)[2].wait()
