"""Sharded update, host side (no GPU): partition of a patch set over ranks, the
ghost regions, and a 2-rank ghost exchange over torch.distributed (gloo)
checked against the oracle's periodic ghost fill."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from paper_2110_01792_gb300 import shard as S


def _layout():
    return I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=3, edges=(8, 16, 24))


def _truth(lay, nf=3, seed=12):
    rng = np.random.Generator(np.random.Philox(seed))
    fields = [np.zeros(lay.field_len) for _ in range(nf)]
    for f in fields:
        for b in range(lay.nbox):
            lay.interior(f, b)[...] = rng.standard_normal(lay.interior(f, b).shape)
    filled = [f.copy() for f in fields]
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    for f in filled:
        O.fill_ghosts(g, f)
    return fields, filled


@pytest.mark.parametrize("nranks", [2, 3, 4])
def test_partition_balanced(nranks):
    lay = _layout()
    owner = S.partition(lay, nranks)
    cells = np.prod(lay.n.astype(np.int64), axis=1)
    per = np.array([cells[owner == r].sum() for r in range(nranks)])
    assert np.all(per > 0) and per.sum() == cells.sum()
    assert np.all(np.abs(per - cells.sum() / nranks) <= cells.max())


def test_ghost_regions_reproduce_the_periodic_fill():
    """Applying every ghost region as a copy reproduces the oracle's ghost fill
    (periodic images, non-conforming neighbours, corners and edges)."""
    lay = _layout()
    fields, filled = _truth(lay)
    S.apply_local(lay, fields, S.ghost_regions(lay))
    for f, t in zip(fields, filled):
        for b in range(lay.nbox):
            assert np.array_equal(lay.full(f, b), lay.full(t, b))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lay = _layout()
        owner = S.partition(lay, world)
        plan = S.exchange_plan(lay, owner)
        fields, filled = _truth(lay)
        # this rank holds only its own patches' interiors; everything else NaN
        local = [np.full(lay.field_len, np.nan) for _ in fields]
        for lf, f in zip(local, fields):
            for b in np.nonzero(owner == rank)[0]:
                lay.interior(lf, b)[...] = lay.interior(f, b)
        S.exchange(lay, local, plan, rank)
        ok = all(np.array_equal(lay.full(lf, b), lay.full(t, b))
                 for lf, t in zip(local, filled) for b in np.nonzero(owner == rank)[0])
        gmax = S.global_max(rank + 1.5)
        results[rank] = (bool(ok), gmax, sum(len(v) for v in plan[rank]["send"].values()))
    finally:
        dist.destroy_process_group()


def test_two_rank_exchange_gloo():
    """Two gloo ranks own complementary halves of the patch set; after the
    exchange every owned patch's ghost layer equals the global periodic fill
    (non-owned data were NaN, so no wrong source can go unnoticed), and the
    max-reduction of the signal speed is the global one."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        ok, gmax, nsend = results[r]
        assert ok and gmax == world + 0.5 and nsend > 0
