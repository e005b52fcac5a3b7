"""Host logic of the spatial domain decomposition (paper_1806_05089_gb300.decomp),
on the CPU: the partition, the exchange plan, and the halo exchange itself,
in one process and over torch.distributed (gloo, world size 2).

Each block's state here is a CPU tensor pair (populations, gauge) cut from a
global periodic field with its halos blanked; after one exchange every halo
must hold the global field's values -- the same schedule code that moves the
library's packed strips between GPUs.
"""
import os
import socket

import numpy as np
import pytest
import torch

from paper_1806_05089_gb300 import decomp

Q = 16


def global_state(nx, ny, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((Q, ny, nx)), rng.standard_normal((3, ny, nx))


def block_state(part, rank, f, g, blank=True):
    ys, xs = part.padded_slices(rank)
    fb = torch.tensor(f[:, ys][:, :, xs])
    gb = torch.tensor(g[:, ys][:, :, xs])
    if blank:
        H = part.halo
        keep_f = fb[:, H:-H, H:-H].clone()
        keep_g = gb[:, H:-H, H:-H].clone()
        fb.fill_(np.nan)
        gb.fill_(np.nan)
        fb[:, H:-H, H:-H] = keep_f
        gb[:, H:-H, H:-H] = keep_g
    return {"f": fb, "g": gb}


def pack(st, rect, buf):
    n = rect.size
    sl = (slice(None), slice(rect.y0, rect.y0 + rect.h), slice(rect.x0, rect.x0 + rect.w))
    buf[:Q * n] = st["f"][sl].reshape(-1)
    buf[Q * n:] = st["g"][sl].reshape(-1)


def unpack(st, rect, buf):
    n = rect.size
    sl = (slice(None), slice(rect.y0, rect.y0 + rect.h), slice(rect.x0, rect.x0 + rect.w))
    st["f"][sl] = buf[:Q * n].reshape(Q, rect.h, rect.w)
    st["g"][sl] = buf[Q * n:].reshape(3, rect.h, rect.w)


def alloc(n):
    return torch.empty((Q + 3) * n, dtype=torch.float64)


@pytest.mark.parametrize("nx,ny,px,py", [(128, 64, 2, 1), (100, 72, 3, 2), (64, 40, 1, 1),
                                         (96, 96, 3, 3)])
def test_blocks_tile_the_grid(nx, ny, px, py):
    part = decomp.Partition(nx, ny, px, py, halo=6, align_x=32, align_y=8)
    cover = np.zeros((ny, nx), dtype=int)
    for r in range(part.size):
        b = part.block(r)
        cover[b.y0:b.y0 + b.h, b.x0:b.x0 + b.w] += 1
        assert part.rank_of(b.bx, b.by) == r
    assert np.all(cover == 1)
    # inner boundaries on the tile grid where the sizes allow it
    if nx % (32 * px) == 0:
        assert all(c % 32 == 0 for c in part.xcuts)


def test_block_narrower_than_halo_is_rejected():
    with pytest.raises(ValueError):
        decomp.Partition(40, 40, 8, 1, halo=6, align_x=1, align_y=1)


@pytest.mark.parametrize("px,py", [(1, 1), (2, 1), (1, 2), (2, 2), (3, 2)])
def test_every_send_has_a_matching_receive(px, py):
    part = decomp.Partition(96, 48, px, py, halo=5, align_x=1, align_y=1)
    for ph in range(2):
        sends, recvs = [], []
        for r in range(part.size):
            phase = part.plan(r)[ph]
            sends += [(r, t.peer, t.tag, t.rect.w, t.rect.h) for t in phase.sends]
            recvs += [(t.peer, r, t.tag, t.rect.w, t.rect.h) for t in phase.recvs]
        assert sorted(sends) == sorted(recvs)


@pytest.mark.parametrize("nx,ny,px,py,halo", [(64, 48, 1, 1, 5), (96, 48, 2, 1, 6),
                                              (64, 64, 1, 2, 4), (96, 72, 2, 2, 6),
                                              (100, 72, 3, 2, 7)])
def test_local_exchange_fills_every_halo(nx, ny, px, py, halo):
    part = decomp.Partition(nx, ny, px, py, halo, align_x=1, align_y=1)
    f, g = global_state(nx, ny)
    blocks = {r: block_state(part, r, f, g) for r in range(part.size)}
    decomp.exchange(part, blocks, pack, unpack, decomp.LocalTransport(), alloc)
    for r, st in blocks.items():
        ref = block_state(part, r, f, g, blank=False)
        assert torch.equal(st["f"], ref["f"]) and torch.equal(st["g"], ref["g"]), r


def test_local_transport_max_is_the_local_value():
    assert decomp.LocalTransport().reduce_max(3.75) == 3.75


def test_halo_width_covers_the_stencil_reach():
    # displacement d moves a departure point at most d nodes; the cubic
    # stencil reaches from floor(departure) - 1 to floor(departure) + 2
    for d in (0.0, 0.4, 2.33, 4.9, 7.0):
        assert decomp.halo_width(d) >= np.floor(d) + 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, px, py, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = decomp.Partition(80, 48, px, py, halo=5, align_x=1, align_y=1)
        f, g = global_state(80, 48, seed=3)
        blocks = {rank: block_state(part, rank, f, g)}
        tr = decomp.TorchDistTransport()
        decomp.exchange(part, blocks, pack, unpack, tr, alloc)
        ref = block_state(part, rank, f, g, blank=False)
        ok = torch.equal(blocks[rank]["f"], ref["f"]) and torch.equal(blocks[rank]["g"], ref["g"])
        # the displacement bound every rank checks its halo against is the
        # maximum over the ranks
        ok = ok and tr.reduce_max(1.5 + 2.25 * rank) == 1.5 + 2.25 * (world - 1)
        out[rank] = int(ok)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
def test_exchange_over_gloo_world_size_2(px, py):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, px, py, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 1, 1: 1}


def test_ensemble_shards_cover_every_grid_once_and_balance_nodes():
    from paper_1806_05089_gb300 import workloads
    nx, ny = workloads.ensemble_sizes(256)
    nodes = np.array(nx) * np.array(ny)
    for world in (1, 2, 4, 8):
        shards = decomp.ensemble_shards(nx, ny, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(256))
        load = [int(nodes[s].sum()) for s in shards]
        # greedy largest-first: no rank exceeds the mean by more than the
        # largest grid
        assert max(load) - min(load) <= nodes.max()
