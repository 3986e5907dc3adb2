"""Sharded update on the GPU: a patch set split over virtual ranks (one shard
context per rank, all on one GPU, halos moved by device copies between
launches) advances bit-for-bit like the whole patch set in one context.

Each rank packs its outgoing halo, the host copies every buffer to the
peer's receive buffer, then each rank unpacks: no kernel ever waits on another
rank, so running the ranks on one GPU is safe."""
import numpy as np
import pytest

from paper_2110_01792_gb300 import inputs as I
from paper_2110_01792_gb300 import shard as S
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_01792_gb300 import qk
    qk.lib()
    return torch


def _problem(flattening=0):
    lay = I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=4, edges=(8, 16, 24))
    prob = I.rhd_lognormal(layout=lay, seed=21)
    rng = np.random.Generator(np.random.Philox(77))
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        v = 0.3 * rng.standard_normal((3,) + rho.shape)
        for d in range(3):
            lay.interior(prob.U[1 + d], b)[...] = rho * v[d]
        lay.interior(prob.U[4], b)[...] += 0.5 * rho * (v ** 2).sum(0)
    prm = dict(prob.params)
    prm["dx"] = 1.0 / 48
    prm["flattening"] = flattening
    return lay, prob, prm


def _to_rank(lay, rlay, owner, rank, arrays, dtype):
    out = []
    for a in arrays:
        r = np.zeros(rlay.field_len)
        for b in np.nonzero(owner == rank)[0]:
            rlay.full(r, b)[...] = lay.full(a, b)
        out.append(r)
    return G.dev(out, dtype)


def _single(lay, prob, prm, prec, steps, dtype):
    from paper_2110_01792_gb300 import qk
    ctx = qk.Context(lay, prm, prec)
    U, R = G.dev(prob.U, dtype), G.dev(prob.R, dtype)
    hist = [ctx.step(U, R, want_dt=True) for _ in range(steps)]
    out = G.host(U) + G.host(R)
    ctx.close()
    return out, hist


def _sharded(lay, prob, prm, prec, steps, nranks, dtype):
    from paper_2110_01792_gb300 import qk
    owner = S.partition(lay, nranks)
    ranks = []
    for r in range(nranks):
        rlay = S.rank_layout(lay, owner, r)
        ctx = qk.Context(rlay, prm, prec, owner=owner, rank=r)
        U = _to_rank(lay, rlay, owner, r, prob.U, dtype)
        R = _to_rank(lay, rlay, owner, r, prob.R, dtype)
        ranks.append((rlay, ctx, S.RankStepper(ctx, U, R)))
    # the halo lists of every rank pair agree in size
    for r, (_, ctx, _) in enumerate(ranks):
        for p, (_, cp, _) in enumerate(ranks):
            if p != r:
                assert ctx.halo_cells(p)[0] == cp.halo_cells(r)[1]
    assert sum(c.num_cells for _, c, _ in ranks) == lay.ncells
    hist = []
    for _ in range(steps):
        res = S.run_local([st for _, _, st in ranks])
        assert len(set(res)) == 1, res
        hist.append(res[0])
    out = [np.zeros(lay.field_len) for _ in range(9)]
    for r, (rlay, ctx, st) in enumerate(ranks):
        got = G.host(st.U) + G.host(st.R)
        for f in range(9):
            for b in np.nonzero(owner == r)[0]:
                lay.interior(out[f], b)[...] = rlay.interior(got[f], b)
        ctx.close()
    return out, hist


@pytest.mark.parametrize("prec,nranks,flat", [(0, 2, 0), (0, 3, 1), (1, 2, 0), (1, 4, 0)])
def test_sharded_step_bit_identical(torch_cuda, prec, nranks, flat):
    """RHD (hydro + N_sub radiation substeps + exchange) for 3 steps on a
    non-conforming periodic patch set: ranks that own Morton-ordered runs of
    patches and trade halos give every cell bit-for-bit the value of the
    single-context qk_step, with identical dt and N_sub (global max of the
    signal speed)."""
    torch = torch_cuda
    dtype = torch.float64 if prec == 0 else torch.float32
    lay, prob, prm = _problem(flat)
    ref, href = _single(lay, prob, prm, prec, 3, dtype)
    got, hgot = _sharded(lay, prob, prm, prec, 3, nranks, dtype)
    assert [(d, int(n)) for d, n in hgot] == [(d, int(n)) for d, n in href]
    assert max(int(n) for _, n in href) >= 2
    for a, b in zip(got, ref):
        assert np.array_equal(G.interior(lay, a), G.interior(lay, b))


def test_sharded_context_refuses_whole_step(torch_cuda):
    """A shard with peers cannot run qk_step / qk_timestep (they would need the
    other ranks' cells); a one-rank shard context can."""
    from paper_2110_01792_gb300 import qk
    lay, prob, prm = _problem()
    owner = S.partition(lay, 2)
    rlay = S.rank_layout(lay, owner, 0)
    ctx = qk.Context(rlay, prm, 0, owner=owner, rank=0)
    U = _to_rank(lay, rlay, owner, 0, prob.U, torch_cuda.float64)
    with pytest.raises(qk.QKError) as e:
        ctx.step(U)
    assert e.value.code == qk.EINVAL
    with pytest.raises(qk.QKError):
        ctx.timestep(U)
    with pytest.raises(qk.QKError):
        ctx.halo_pack(0, U, U[0])  # this rank is not its own peer
    with pytest.raises(qk.QKError):
        ctx.set_timestep(0.0)
    ctx.close()
    one = np.zeros(lay.nbox, dtype=np.int32)
    ctx = qk.Context(lay, prm, 0, owner=one, rank=0)
    dU = G.dev(prob.U)
    ctx.step(dU)
    ctx.close()


@pytest.mark.parametrize("nranks,flat,bcs", [(2, 1, None), (3, 0, "mixed")])
def test_overlapped_sharded_step_bit_identical(torch_cuda, nranks, flat, bcs):
    """Overlap of the halo transfer with the stage work: every stage runs on
    the interior tiles (no remotely filled ghost cell within 4 cells) before
    the halo moves and on the boundary tiles after; the result is bit for bit
    the single-context qk_step, with flattening and with non-periodic faces.
    Every rank has both kinds of tiles."""
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    lay, prob, prm = _overlap_problem(flat)
    U, R = prob.U, prob.R
    if bcs:
        # outflow / Dirichlet on x, Dirichlet / reflecting on y, reflecting z;
        # the Dirichlet states are whatever the ghost cells hold (zeros are
        # not physical, so the interior state is copied outward first)
        prm = dict(prm, bc_lo=(2, 3, 1), bc_hi=(3, 1, 1))
        U, R = _frozen_ghosts(lay, U, R)
    ref, href = _single_bc(lay, U, R, prm, 3)
    owner = (lay.lo[:, 0] // 32 * nranks // 4).astype(np.int32)
    ranks = []
    for r in range(nranks):
        rlay = S.rank_layout(lay, owner, r)
        ctx = qk.Context(rlay, prm, 0, owner=owner, rank=r)
        ni, nb = ctx.tile_counts()
        assert ni > 0 and nb > 0, (r, ni, nb)
        dU = _to_rank(lay, rlay, owner, r, U, torch.float64)
        dR = _to_rank(lay, rlay, owner, r, R, torch.float64)
        if bcs:
            ctx.set_dirichlet(dU, dR)
        ranks.append((rlay, ctx, S.RankStepper(ctx, dU, dR, overlap=True)))
    hist = [S.run_local([st for _, _, st in ranks])[0] for _ in range(3)]
    assert [(a, int(b)) for a, b in hist] == [(a, int(b)) for a, b in href]
    for r, (rlay, ctx, st) in enumerate(ranks):
        got = G.host(st.U) + G.host(st.R)
        for f in range(9):
            for b in np.nonzero(owner == r)[0]:
                assert np.array_equal(rlay.interior(got[f], b), lay.interior(ref[f], b))
        ctx.close()


def _overlap_problem(flattening):
    """Eight 32^3 patches over 128 x 64 x 32: patches wide enough that tiles
    more than 4 cells from a rank border exist (interior tiles)."""
    lo = [[x, y, 0] for y in (0, 32) for x in range(0, 128, 32)]
    lay = I.make_layout(lo, [[32, 32, 32]] * len(lo), (128, 64, 32), 4)
    prob = I.rhd_lognormal(layout=lay, seed=23)
    rng = np.random.Generator(np.random.Philox(78))
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        v = 0.3 * rng.standard_normal((3,) + rho.shape)
        for d in range(3):
            lay.interior(prob.U[1 + d], b)[...] = rho * v[d]
        lay.interior(prob.U[4], b)[...] += 0.5 * rho * (v ** 2).sum(0)
    prm = dict(prob.params, dx=1.0 / 128, flattening=flattening)
    return lay, prob, prm


def _frozen_ghosts(lay, U, R):
    """Every ghost cell takes the value of the nearest interior cell of its
    patch: a physical state for the ghost cells beyond Dirichlet faces (which
    each patch records for itself)."""
    out = []
    g = lay.ng
    for f in U + R:
        a = f.copy()
        for b in range(lay.nbox):
            full = lay.full(a, b)
            n = lay.n[b]
            iz = np.clip(np.arange(n[2] + 2 * g) - g, 0, n[2] - 1) + g
            iy = np.clip(np.arange(n[1] + 2 * g) - g, 0, n[1] - 1) + g
            ix = np.clip(np.arange(n[0] + 2 * g) - g, 0, n[0] - 1) + g
            full[...] = full[np.ix_(iz, iy, ix)]
        out.append(a)
    return out[:5], out[5:]


def _single_bc(lay, U, R, prm, steps):
    from paper_2110_01792_gb300 import qk
    ctx = qk.Context(lay, prm, 0)
    dU, dR = G.dev(U), G.dev(R)
    if 3 in tuple(prm.get("bc_lo", ())) + tuple(prm.get("bc_hi", ())):
        ctx.set_dirichlet(dU, dR)
    hist = [ctx.step(dU, dR, want_dt=True) for _ in range(steps)]
    out = G.host(dU) + G.host(dR)
    ctx.close()
    return out, hist


def _sharded_overlap(lay, prob_U, prob_R, prm, prec, steps, owner, dtype):
    from paper_2110_01792_gb300 import qk
    nranks = int(owner.max()) + 1
    ranks = []
    for r in range(nranks):
        rlay = S.rank_layout(lay, owner, r)
        ctx = qk.Context(rlay, prm, prec, owner=owner, rank=r)
        U = _to_rank(lay, rlay, owner, r, prob_U, dtype)
        R = _to_rank(lay, rlay, owner, r, prob_R, dtype)
        ranks.append((rlay, ctx, S.RankStepper(ctx, U, R, overlap=True)))
    hist = [S.run_local([st for _, _, st in ranks])[0] for _ in range(steps)]
    out = [np.zeros(lay.field_len) for _ in range(9)]
    for r, (rlay, ctx, st) in enumerate(ranks):
        got = G.host(st.U) + G.host(st.R)
        for f in range(9):
            for b in np.nonzero(owner == r)[0]:
                lay.interior(out[f], b)[...] = rlay.interior(got[f], b)
        ctx.close()
    return out, hist


@pytest.mark.parametrize("nranks,layout", [(2, "tiling"), (3, "tiling"), (2, "slabs")])
def test_sharded_step_matches_oracle(torch_cuda, nranks, layout):
    """The sharded update checked against the FP64 oracle itself (not against
    the single-context GPU path): virtual ranks with overlapped halo
    transfers and the fused exchange advance 3 RHD steps (hydro, N_sub
    radiation substeps, exchange); every interior cell matches the oracle's
    single-grid step to 1e-10 (max relative error, RMS floor), with the same
    dt and N_sub."""
    import oracle as O
    torch = torch_cuda
    if layout == "tiling":
        lay, prob, prm = _problem(0)
        owner = S.partition(lay, nranks)
    else:
        lay, prob, prm = _overlap_problem(0)
        owner = (lay.lo[:, 0] // 32 * nranks // 4).astype(np.int32)
    got, hist = _sharded_overlap(lay, prob.U, prob.R, prm, 0, 3, owner, torch.float64)
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    p = O.make_params(**prm)
    Uo = [a.copy() for a in prob.U]
    Ro = [a.copy() for a in prob.R]
    O.set_threads(8)
    try:
        for dt, nsub in hist:
            rc, ts, _ = O.step(g, p, Uo, Ro)
            assert rc == 0 and int(ts[1]) == int(nsub) and abs(ts[0] - dt) <= 1e-13 * dt
    finally:
        O.set_threads(1)
    assert max(int(n) for _, n in hist) >= 2
    err = G.max_rel_err(lay, got, Uo + Ro)
    assert max(err) <= 1e-10, err
