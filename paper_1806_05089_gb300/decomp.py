"""Spatial domain decomposition of one periodic PonD grid.

Eq. advection reads only the state at t - dt, so a grid split into
px x py blocks advances block by block: each block's context holds its
interior plus a halo of width H on every side, the step updates the interior
only (``pond_set_interior``), and between steps each block refreshes its halo
from its neighbours' interiors -- one exchange per step, whatever the number
of predictor-corrector passes.  H must exceed the largest displacement of a
step plus the reach of the cubic stencil: H >= ceil(max(|u| + c_max
sqrt(theta)) dt) + 3 (the +3: the stencil spans floor(departure) - 1 ..
floor(departure) + 2, and one node of slack for the pass gauges).

The exchange runs in two phases, so the corner halos need no messages of
their own: first the x-halos (left and right strips of the interior rows),
then the y-halos over the full padded width (which by then carries the
x-halos).  A peer may be the block itself (one block along an axis: the
periodic wrap) or the same block on both sides (two blocks along an axis).

Messages are moved by a transport: ``TorchDistTransport`` (one block per
rank, ``torch.distributed`` point-to-point, NCCL between GPUs or gloo on the
CPU) or ``LocalTransport`` (all blocks in one process, messages handed over
directly; used to check a split against the single-grid step on one GPU).
The strips are packed and unpacked by the library (``pond_pack_rect`` /
``pond_unpack_rect``, the stored representation, so a split run is
bit-identical to the single-grid run when the block origins fall on the
staged kernel's tile grid).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------------ partition

@dataclass(frozen=True)
class Block:
    rank: int
    bx: int
    by: int
    x0: int  # interior origin in global coordinates
    y0: int
    w: int   # interior size
    h: int


@dataclass(frozen=True)
class Rect:
    x0: int  # in the block's padded local coordinates
    y0: int
    w: int
    h: int

    @property
    def size(self) -> int:
        return self.w * self.h


@dataclass(frozen=True)
class Transfer:
    peer: int
    rect: Rect
    tag: int


@dataclass
class Phase:
    sends: list = field(default_factory=list)  # Transfer, in issue order
    recvs: list = field(default_factory=list)


def split(n: int, parts: int, align: int) -> list:
    """Block boundaries of n nodes in `parts` blocks, as equal as possible,
    each inner boundary a multiple of `align` when that leaves every block
    non-empty (else plain equal parts)."""
    cuts = [0]
    for i in range(1, parts):
        c = round(i * n / parts / align) * align
        cuts.append(c)
    cuts.append(n)
    if any(b <= a for a, b in zip(cuts, cuts[1:])):
        cuts = [i * n // parts for i in range(parts)] + [n]
    return cuts


class Partition:
    """px x py blocks of an nx x ny periodic grid with halo width `halo`.
    Rank r owns block (bx, by) = (r % px, r // px).  Inner block boundaries
    are aligned to (align_x, align_y) where possible."""

    def __init__(self, nx: int, ny: int, px: int, py: int, halo: int,
                 align_x: int = 32, align_y: int = 8):
        if px < 1 or py < 1 or halo < 1:
            raise ValueError("px, py and the halo must be positive")
        self.nx, self.ny, self.px, self.py, self.halo = nx, ny, px, py, halo
        self.xcuts = split(nx, px, align_x)
        self.ycuts = split(ny, py, align_y)
        for cuts in (self.xcuts, self.ycuts):
            if min(b - a for a, b in zip(cuts, cuts[1:])) < halo:
                raise ValueError("a block is narrower than the halo (%d); use fewer blocks" % halo)

    @property
    def size(self) -> int:
        return self.px * self.py

    def rank_of(self, bx: int, by: int) -> int:
        return (by % self.py) * self.px + (bx % self.px)

    def block(self, rank: int) -> Block:
        bx, by = rank % self.px, rank // self.px
        x0, x1 = self.xcuts[bx], self.xcuts[bx + 1]
        y0, y1 = self.ycuts[by], self.ycuts[by + 1]
        return Block(rank, bx, by, x0, y0, x1 - x0, y1 - y0)

    def padded_shape(self, rank: int):
        b = self.block(rank)
        return b.h + 2 * self.halo, b.w + 2 * self.halo  # (ny, nx)

    def plan(self, rank: int):
        """The two exchange phases of `rank`: sends of interior strips and
        receives into halo strips, local padded coordinates.  In each phase
        the sends go to (left, right) or (down, up) and the receives come
        from (right, left) or (up, down), in that order, with tags naming the
        receiving side, so messages between one pair of ranks match in issue
        order (NCCL) and by tag (gloo) alike."""
        H = self.halo
        b = self.block(rank)
        left, right = self.rank_of(b.bx - 1, b.by), self.rank_of(b.bx + 1, b.by)
        down, up = self.rank_of(b.bx, b.by - 1), self.rank_of(b.bx, b.by + 1)
        W = b.w + 2 * H
        px = Phase(
            sends=[Transfer(left, Rect(H, H, H, b.h), 0),          # -> left's right halo
                   Transfer(right, Rect(b.w, H, H, b.h), 1)],      # -> right's left halo
            recvs=[Transfer(right, Rect(H + b.w, H, H, b.h), 0),   # right's left strip
                   Transfer(left, Rect(0, H, H, b.h), 1)])         # left's right strip
        py = Phase(
            sends=[Transfer(down, Rect(0, H, W, H), 2),            # -> down's top halo
                   Transfer(up, Rect(0, b.h, W, H), 3)],           # -> up's bottom halo
            recvs=[Transfer(up, Rect(0, H + b.h, W, H), 2),
                   Transfer(down, Rect(0, 0, W, H), 3)])
        return [px, py]

    def padded_slices(self, rank: int):
        """Global (periodic) row and column indices of rank's padded block."""
        b = self.block(rank)
        H = self.halo
        ys = np.arange(b.y0 - H, b.y0 + b.h + H) % self.ny
        xs = np.arange(b.x0 - H, b.x0 + b.w + H) % self.nx
        return ys, xs


def halo_width(max_displacement: float) -> int:
    """Smallest safe halo for a step whose particles move at most
    `max_displacement` nodes."""
    return int(math.ceil(max_displacement)) + 3


# ------------------------------------------------------------------ transports

class LocalTransport:
    """All blocks live in this process: a receive takes the matching send's
    buffer (same source, destination and tag)."""

    def reduce_max(self, value: float) -> float:
        """The maximum over all blocks of a per-process value: this process
        holds every block."""
        return float(value)

    def run(self, ops):
        """ops: list of (rank, phase, send_buffers, recv_buffers) for every
        block; fills the receive buffers."""
        posted = {}
        for rank, phase, sbufs, _ in ops:
            for t, buf in zip(phase.sends, sbufs):
                posted[(rank, t.peer, t.tag)] = buf
        for rank, phase, _, rbufs in ops:
            for t, buf in zip(phase.recvs, rbufs):
                buf.copy_(posted[(t.peer, rank, t.tag)])


class TorchDistTransport:
    """One block per rank; torch.distributed point-to-point (NCCL or gloo).
    Sends and receives of a phase are posted together and waited for."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def reduce_max(self, value: float) -> float:
        """The maximum of a per-rank value over the ranks (an all-reduce;
        on the GPU for NCCL, on the host for gloo), so that every rank takes
        the same decision from it."""
        import torch
        backend = self.dist.get_backend(self.group)
        dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else None
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def run(self, ops):
        dist = self.dist
        reqs = []
        for rank, phase, sbufs, rbufs in ops:
            # a block that is its own neighbour (one block along an axis)
            # copies locally; the backends do not send to self
            own = {t.tag: buf for t, buf in zip(phase.sends, sbufs) if t.peer == rank}
            p2p = [dist.P2POp(dist.isend, buf, t.peer, self.group, t.tag)
                   for t, buf in zip(phase.sends, sbufs) if t.peer != rank]
            p2p += [dist.P2POp(dist.irecv, buf, t.peer, self.group, t.tag)
                    for t, buf in zip(phase.recvs, rbufs) if t.peer != rank]
            for t, buf in zip(phase.recvs, rbufs):
                if t.peer == rank:
                    buf.copy_(own[t.tag])
            if p2p:
                reqs += dist.batch_isend_irecv(p2p)
        for r in reqs:
            r.wait()


def exchange(part: Partition, blocks: dict, pack, unpack, transport, alloc):
    """One halo refresh of the local blocks {rank: state}: for each phase,
    pack every send strip (pack(state, rect, buf)), move the messages, unpack
    every received strip (unpack(state, rect, buf)).  alloc(n) makes a
    message buffer of n strip nodes."""
    plans = {r: part.plan(r) for r in blocks}
    for ph in range(2):
        ops = []
        for r, st in blocks.items():
            phase = plans[r][ph]
            sbufs = [alloc(t.rect.size) for t in phase.sends]
            for t, buf in zip(phase.sends, sbufs):
                pack(st, t.rect, buf)
            rbufs = [alloc(t.rect.size) for t in phase.recvs]
            ops.append((r, phase, sbufs, rbufs))
        transport.run(ops)
        for r, phase, _, rbufs in ops:
            for t, buf in zip(phase.recvs, rbufs):
                unpack(blocks[r], t.rect, buf)


# ------------------------------------------------------------------ PonD blocks

class DecomposedSim:
    """One periodic nx x ny PonD grid split into px x py blocks, each a
    library context on the current CUDA device with its interior set.
    ``ranks`` are the blocks this process owns (all of them with
    LocalTransport, its own rank with TorchDistTransport).  The staged
    kernel runs the blocks (tile_rows fixes its tile; block origins are
    aligned to it)."""

    def __init__(self, nx, ny, px, py, halo, precision=None, ranks=None, transport=None,
                 tile_rows=8, stream=None, **cfg):
        import torch
        from . import pond
        self.torch = torch
        self.pond = pond
        if precision is None:
            precision = pond.POND_FP64
        self.part = Partition(nx, ny, px, py, halo, align_x=32, align_y=tile_rows)
        self.ranks = list(range(self.part.size)) if ranks is None else list(ranks)
        self.transport = transport or LocalTransport()
        self.sims = {}
        for r in self.ranks:
            pny, pnx = self.part.padded_shape(r)
            s = pond.Sim(pnx, pny, precision, stream=stream, kernel=pond.POND_KERNEL_STAGED,
                         tile_rows=tile_rows, **cfg)
            b = self.part.block(r)
            pond.pond_set_interior(s.ctx, 0, halo, halo, b.w, b.h)
            self.sims[r] = s
        self.Q = next(iter(self.sims.values())).Q

    def close(self):
        for s in self.sims.values():
            s.close()
        self.sims = {}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, rho, ux, uy, T):
        """Global fields [ny][nx]: every block takes its padded window (the
        periodic wrap fills the outer halos)."""
        for r, s in self.sims.items():
            ys, xs = self.part.padded_slices(r)
            sub = lambda a: np.ascontiguousarray(a[np.ix_(ys, xs)])
            s.set_state(sub(rho), sub(ux), sub(uy), sub(T))

    def _pack(self, sim, rect, buf):
        self.pond.pond_pack_rect(sim.ctx, 0, rect.x0, rect.y0, rect.w, rect.h, buf, q=self.Q)

    def _unpack(self, sim, rect, buf):
        self.pond.pond_unpack_rect(sim.ctx, 0, rect.x0, rect.y0, rect.w, rect.h, buf, q=self.Q)

    def _alloc(self, n):
        return self.torch.empty((self.Q + 3) * n, dtype=self.torch.float64, device="cuda")

    def max_displacement(self) -> float:
        """The largest displacement of one step over the whole grid: the
        local blocks' bound, reduced over the ranks by the transport."""
        local = max(self.pond.pond_max_displacement(s.ctx, 0) for s in self.sims.values())
        return self.transport.reduce_max(local)

    def step(self, nsteps: int = 1, check: bool = True):
        """nsteps steps, each one halo exchange then one step of every local
        block.  With check, the displacement bound (reduced over all ranks,
        so that every rank refuses the same step) is verified against the
        halo before each step."""
        stats = []
        for _ in range(nsteps):
            if check:
                d = self.max_displacement()
                if halo_width(d) > self.part.halo:
                    raise RuntimeError("displacement %.2f needs a halo of %d > %d"
                                       % (d, halo_width(d), self.part.halo))
            self.torch.cuda.synchronize()
            exchange(self.part, self.sims, self._pack, self._unpack, self.transport, self._alloc)
            self.torch.cuda.synchronize()
            stats.append({r: s.step(1) for r, s in self.sims.items()})
        return stats

    def gather(self):
        """(rho, ux, uy, T) of the local blocks' interiors placed into global
        arrays (zeros where another process owns the block)."""
        nx, ny = self.part.nx, self.part.ny
        out = [np.zeros((ny, nx)) for _ in range(4)]
        H = self.part.halo
        for r, s in self.sims.items():
            b = self.part.block(r)
            m = s.moments()
            for o, a in zip(out, m):
                o[b.y0:b.y0 + b.h, b.x0:b.x0 + b.w] = a[H:H + b.h, H:H + b.w]
        return tuple(out)

    def gather_state(self):
        """Populations and gauge of the interiors, global [Q][ny][nx] etc."""
        nx, ny = self.part.nx, self.part.ny
        f = np.zeros((self.Q, ny, nx))
        g = [np.zeros((ny, nx)) for _ in range(3)]
        H = self.part.halo
        for r, s in self.sims.items():
            b = self.part.block(r)
            st = s.state()
            f[:, b.y0:b.y0 + b.h, b.x0:b.x0 + b.w] = st.f[:, H:H + b.h, H:H + b.w]
            for o, a in zip(g, (st.ux, st.uy, st.T)):
                o[b.y0:b.y0 + b.h, b.x0:b.x0 + b.w] = a[H:H + b.h, H:H + b.w]
        return f, g


# ------------------------------------------------------------------ ensembles

def ensemble_shards(nx, ny, world: int):
    """Whole grids of an ensemble assigned to `world` ranks (no data is
    exchanged between grids, so each rank runs its share as one batched
    context): largest grid first, each to the rank with the fewest nodes so
    far.  Returns one list of grid indices per rank, each in ascending
    order."""
    if world < 1:
        raise ValueError("world must be positive")
    sizes = [int(a) * int(b) for a, b in zip(nx, ny)]
    load = [0] * world
    shards = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        shards[r].append(i)
        load[r] += sizes[i]
    return [sorted(s) for s in shards]
