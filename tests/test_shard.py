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


# ------------------------------------- step composer over torch.distributed ---
class _Params:
    hydro_only = 0


class FakeShardCtx:
    """Stand-in for one rank's library context with the same methods, in numpy
    on the host: ghost fills and halos follow ``exchange_plan``; the stages are
    simple neighbour stencils that read the ghost cells (so a missing or wrong
    halo changes the result); the timestep is a fixed function of the speed."""

    def __init__(self, lay, owner, rank):
        self.lay, self.owner, self.rank = lay, owner, rank
        self.nranks = int(owner.max()) + 1
        self.plan = S.exchange_plan(lay, owner)[rank]
        self.own = np.nonzero(owner == rank)[0]
        self.params = _Params()
        # patch-level stand-in for the interior / boundary tile split: a patch
        # is "boundary" when any of its ghost regions comes from another rank
        remote = {r[0] for regs in self.plan["recv"].values() for r in regs}
        self.parts = {0: self.own, 1: np.array([b for b in self.own if b not in remote]),
                      2: np.array([b for b in self.own if b in remote])}
        self.part = 0

    def set_tile_part(self, part):
        self.part = part

    @staticmethod
    def _np(fields):
        return [f.numpy() for f in fields]

    def halo_cells(self, p):
        vol = lambda regs: sum(r[4][0] * r[4][1] * r[4][2] for r in regs)
        return vol(self.plan["send"].get(p, [])), vol(self.plan["recv"].get(p, []))

    def fill_ghosts(self, fields, first=0):
        S.apply_local(self.lay, self._np(fields), self.plan["local"])

    def halo_pack(self, p, fields, buf, first=0):
        buf.numpy()[...] = S.pack(self.lay, self._np(fields), self.plan["send"][p])

    def halo_unpack(self, p, fields, buf, first=0):
        S.unpack(self.lay, self._np(fields), self.plan["recv"][p], buf.numpy())

    def signal_speed(self, U):
        return float(max(np.abs(self.lay.interior(U[1].numpy(), b)).max() for b in self.own))

    def set_timestep(self, smax):
        return 0.01 / smax, 3, 0.004 / smax, smax

    def _lap(self, a, b, rho=None):
        g = self.lay.ng
        v = self.lay.full(a, b)
        n = self.lay.n[b]
        c = lambda dz, dy, dx: v[g + dz:g + dz + n[2], g + dy:g + dy + n[1], g + dx:g + dx + n[0]]
        out = c(0, 0, 1) + c(0, 0, -1) + c(0, 1, 0) + c(0, -1, 0) + c(1, 0, 0) + c(-1, 0, 0) - 6 * c(0, 0, 0)
        if rho is not None:
            w = self.lay.full(rho, b)
            out = out + 0.1 * (w[g:g + n[2], g:g + n[1], g + 2:g + 2 + n[0]] - w[g:g + n[2], g:g + n[1], g - 2:g - 2 + n[0]])
        return out

    def _stage(self, stage, A0, A1, Aout, dt, rho=None):
        src = A0 if stage == 1 else A1
        for f in range(len(A0)):
            a0, s, o = A0[f].numpy(), src[f].numpy(), Aout[f].numpy()
            for b in self.parts[self.part]:
                upd = self.lay.interior(s, b) + dt * self._lap(s, b, rho)
                self.lay.interior(o, b)[...] = upd if stage == 1 else 0.5 * self.lay.interior(a0, b) + 0.5 * upd

    def hydro_stage(self, stage, U0, U1, Uout, dt):
        self._stage(stage, U0, U1, Uout, dt)

    def rad_stage(self, stage, R0, R1, Rout, rho, dt):
        self._stage(stage, R0, R1, Rout, dt, rho.numpy())

    def exchange(self, U, R, dt, patches=None):
        for b in self.own if patches is None else patches:
            e, er = self.lay.interior(U[4].numpy(), b), self.lay.interior(R[0].numpy(), b)
            d = dt * (er - e)
            e += d
            er -= d

    def rad_stage2_exchange(self, R0, R1, Rout, U, dt):
        # stage 2, then the per-cell exchange on the same tile part
        self._stage(2, R0, R1, Rout, dt, U[0].numpy())
        self.exchange(U, Rout, dt, self.parts[self.part])


def _composer_layout():
    """Regular 8^3 patches over 48 x 16 x 16 (periodic), split into x-slabs
    of 24 cells per rank: each rank has patches with and without remote
    neighbours."""
    lo = [[x, y, z] for z in (0, 8) for y in (0, 8) for x in range(0, 48, 8)]
    return I.make_layout(lo, [[8, 8, 8]] * len(lo), (48, 16, 16), 3)


def _composer_owner(lay, world):
    return (lay.lo[:, 0] * world // 48).astype(np.int32)


def _composer_fields(lay, owner, rank):
    import torch
    rng = np.random.Generator(np.random.Philox(31))
    full = [rng.standard_normal(lay.field_len) for _ in range(9)]
    rlay = S.rank_layout(lay, owner, rank)
    out = []
    for f in full:
        r = np.full(rlay.field_len, np.nan)
        for b in np.nonzero(owner == rank)[0]:
            rlay.interior(r, b)[...] = lay.interior(f, b)
        out.append(torch.from_numpy(r))
    return rlay, out[:5], out[5:]


def _composer_run(lay, owner, rank, steps, driver, overlap=False):
    rlay, U, R = _composer_fields(lay, owner, rank)
    st = S.RankStepper(FakeShardCtx(rlay, owner, rank), U, R, overlap=overlap)
    hist = [driver(st) for _ in range(steps)]
    res = {}
    for b in np.nonzero(owner == rank)[0]:
        res[int(b)] = np.stack([rlay.interior(f.numpy(), b) for f in st.U + st.R])
    return res, hist


def _composer_worker(rank, world, port, results, overlap):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lay = _composer_layout()
        owner = _composer_owner(lay, world)
        ctx = FakeShardCtx(S.rank_layout(lay, owner, rank), owner, rank)
        assert len(ctx.parts[1]) > 0 and len(ctx.parts[2]) > 0
        res, hist = _composer_run(lay, owner, rank, 2, S.run_distributed, overlap)
        results[rank] = (res, hist)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("overlap", [False, True])
def test_step_composer_over_gloo_matches_one_rank(overlap):
    """The per-rank step generator driven by ``run_distributed`` on 2 gloo ranks
    (all-reduce for the speed, isend / irecv of packed halos, ghosts NaN
    until filled) gives bit-for-bit the one-rank result of ``run_local`` with
    the same stencil stages: every ghost fill of every stage and substep saw
    the right neighbour data and the global timestep.  With overlap, each
    stage runs on the patches without remote ghosts before the transfer and on
    the others after it (NaN ghosts would leak into any early launch that
    needed the halo)."""
    import torch.multiprocessing as mp
    lay = _composer_layout()
    one = np.zeros(lay.nbox, dtype=np.int32)
    ref, href = _composer_run(lay, one, 0, 2, lambda st: S.run_local([st])[0])
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_composer_worker, args=(r, world, port, results, overlap))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = {}
    for r in range(world):
        res, hist = results[r]
        assert hist == href
        got.update(res)
    assert sorted(got) == sorted(ref)
    for b in ref:
        assert np.all(np.isfinite(got[b]))
        assert np.array_equal(got[b], ref[b])
