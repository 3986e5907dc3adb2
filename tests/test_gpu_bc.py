"""GPU parity of the non-periodic boundaries, the Minerbo and Eddington
closures and the radiation source term: the CUDA path (through the C ABI)
against the FP64 oracle on the same seeded inputs.  Ghost fills bit-exact;
FP64 stages <= 1e-12 and 5 full steps <= 1e-10 per cell (floor = the field's
RMS); the radiation pressure tube of Sec. 3.3.1 within the paper's 0.2 %."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from paper_2110_01792_gb300 import shard as S
from tests import gpu_util as G
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL_STAGE = 1e-12
TOL_STEPS = 1e-10
PER, REF, OUT, DIR = 0, 1, 2, 3
PRM = dict(gamma=5.0 / 3.0, cfl=0.3, c=20.0, chat=4.0, kappa_P=2.0, kappa_R=3.0, a_r=1.0,
           c_v=1.5, dx=0.1)
BCS = {
    "reflect_x_outflow_y": ((REF, OUT, PER), (REF, OUT, PER)),
    "dirichlet_x_reflect_y_outflow_z": ((DIR, REF, OUT), (DIR, REF, OUT)),
    "mixed_faces": ((OUT, DIR, REF), (DIR, REF, REF)),
    "all_dirichlet": ((DIR, DIR, DIR), (DIR, DIR, DIR)),
}


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


def _grid(lay):
    return O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)


def _ctx(lay, prm, prec=0, **kw):
    from paper_2110_01792_gb300 import qk
    return qk.Context(lay, prm, prec, **kw)


def _state_with_boundary(lay, bc_lo, bc_hi, seed):
    """Random RHD state on the domain extended by ng cells; the interior
    cells take the middle, and every ghost cell takes the extended state at
    its position (periodic axes wrapped), so that the Dirichlet states are a
    consistent function of position."""
    ng = lay.ng
    n = lay.dom_n
    ext = P.random_state(tuple(m + 2 * ng for m in n), seed)
    fields = I.zeros(lay, 9)
    for f, e in zip(fields, ext):
        for b in range(lay.nbox):
            full = lay.full(f, b)
            idx = []
            for d in range(3):
                x = np.arange(lay.lo[b][d] - ng, lay.lo[b][d] + lay.n[b][d] + ng)
                if bc_lo[d] == PER:
                    x = np.mod(x, n[d])
                idx.append(x + ng)
            full[...] = e[np.ix_(idx[2], idx[1], idx[0])]
    return fields[:5], fields[5:]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(BCS))
def test_ghost_fill_with_boundaries_bit_exact(torch_cuda, name, prec):
    """Every ghost cell (faces, edges, corners; two patches of unequal width;
    a 16-patch tiling) equals the oracle's boundary-resolved value bit for
    bit: mirror images with m and F negated along the reflecting axis,
    clamped cells, Dirichlet states recorded by qk_set_dirichlet."""
    torch = torch_cuda
    bc_lo, bc_hi = BCS[name]
    for lay in (P.two_patches((11, 9, 7)),
                I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=4, edges=(8, 16, 24))):
        U, R = _state_with_boundary(lay, bc_lo, bc_hi, seed=3)
        if prec == 1:
            U = [a.astype(np.float32).astype(np.float64) for a in U]
            R = [a.astype(np.float32).astype(np.float64) for a in R]
        prm = dict(PRM, bc_lo=bc_lo, bc_hi=bc_hi)
        g, p = _grid(lay), O.make_params(**prm)
        if DIR in bc_lo + bc_hi:
            assert O.set_dirichlet(g, p, U, R) == 0
        Ur, Rr = [a.copy() for a in U], [a.copy() for a in R]
        assert O.fill_ghosts_bc(g, p, Ur, 0) == 0
        assert O.fill_ghosts_bc(g, p, Rr, 5) == 0
        ctx = _ctx(lay, prm, prec)
        dt = torch.float64 if prec == 0 else torch.float32
        dU, dR = G.dev(U, dt), G.dev(R, dt)
        if DIR in bc_lo + bc_hi:
            ctx.set_dirichlet(dU, dR)
        # wipe every ghost cell on the device, then fill
        mask = np.zeros(lay.field_len, dtype=bool)
        for b in range(lay.nbox):
            lay.interior(mask, b)[...] = True
        m = torch.from_numpy(mask).cuda()
        for t in dU + dR:
            t.masked_fill_(~m, -123.0)
        ctx.fill_ghosts(dU, 0)
        ctx.fill_ghosts(dR, 5)
        torch.cuda.synchronize()
        for got, ref in zip(G.host(dU) + G.host(dR), Ur + Rr):
            for b in range(lay.nbox):
                assert np.array_equal(lay.full(got, b), lay.full(ref, b)), (name, b)
        ctx.close()


def _oracle_steps(lay, prm, U, R, n, src=None):
    g, p = _grid(lay), O.make_params(**prm)
    U, R = [a.copy() for a in U], [a.copy() for a in R]
    if DIR in tuple(prm.get("bc_lo", ())) + tuple(prm.get("bc_hi", ())):
        assert O.set_dirichlet(g, p, U, R) == 0
    hist = []
    for _ in range(n):
        rc, ts, _ = O.step(g, p, U, R, src=src)
        assert rc == 0
        hist.append((ts[0], ts[1]))
    return U, R, hist


def _gpu_steps(lay, prm, U, R, n, prec=0, src=None):
    torch = pytest.importorskip("torch")
    ctx = _ctx(lay, prm, prec)
    dt = torch.float64 if prec == 0 else torch.float32
    dU, dR = G.dev(U, dt), G.dev(R, dt)
    if DIR in tuple(prm.get("bc_lo", ())) + tuple(prm.get("bc_hi", ())):
        ctx.set_dirichlet(dU, dR)
    dsrc = G.dev([src], dt)[0] if src is not None else None
    if dsrc is not None:
        ctx.set_source(dsrc)
    hist = [ctx.step(dU, dR, want_dt=True) for _ in range(n)]
    torch.cuda.synchronize()
    st = ctx.status()
    ctx.close()
    return G.host(dU), G.host(dR), hist, st


def _check_hist(hg, hr):
    for (dg, ng_), (dr, nr) in zip(hg, hr):
        assert abs(dg - dr) <= 1e-13 * dr and int(ng_) == int(nr)


@pytest.mark.parametrize("name,recon,flat", [("reflect_x_outflow_y", 0, 0),
                                             ("dirichlet_x_reflect_y_outflow_z", 1, 0),
                                             ("mixed_faces", 0, 1), ("all_dirichlet", 0, 0)])
def test_rhd_steps_with_boundaries_match_oracle(torch_cuda, name, recon, flat):
    """5 full RHD steps (hydro, N_sub radiation substeps, exchange) on two
    patches with non-periodic faces agree with the oracle to 1e-10 per cell;
    dt and N_sub agree; no Newton failure."""
    bc_lo, bc_hi = BCS[name]
    lay = P.two_patches((12, 9, 8))
    U, R = _state_with_boundary(lay, bc_lo, bc_hi, seed=11)
    prm = dict(PRM, bc_lo=bc_lo, bc_hi=bc_hi, recon=recon, flattening=flat)
    Ug, Rg, hg, st = _gpu_steps(lay, prm, U, R, 5)
    Ur, Rr, hr = _oracle_steps(lay, prm, U, R, 5)
    assert st[0] == 0, st
    _check_hist(hg, hr)
    e = G.max_rel_err(lay, Ug + Rg, Ur + Rr)
    assert max(e) <= TOL_STEPS, e


def test_mixed_precision_with_boundaries(torch_cuda):
    """FP32-mixed with reflecting and Dirichlet faces: relative L1 error in
    rho, E and E_r against the FP64 oracle <= 1e-5 after 5 steps."""
    bc_lo, bc_hi = BCS["dirichlet_x_reflect_y_outflow_z"]
    lay = P.two_patches((12, 9, 8))
    U, R = _state_with_boundary(lay, bc_lo, bc_hi, seed=12)
    U = [a.astype(np.float32).astype(np.float64) for a in U]
    R = [a.astype(np.float32).astype(np.float64) for a in R]
    prm = dict(PRM, bc_lo=bc_lo, bc_hi=bc_hi)
    Ug, Rg, _, st = _gpu_steps(lay, prm, U, R, 5, prec=1)
    Ur, Rr, _ = _oracle_steps(lay, prm, U, R, 5)
    assert st[0] == 0, st
    l1 = G.rel_l1(lay, [Ug[0], Ug[4], Rg[0]], [Ur[0], Ur[4], Rr[0]])
    assert max(l1) <= 1e-5, l1


@pytest.mark.parametrize("closure", [1, 2], ids=["minerbo", "eddington"])
def test_closures_match_oracle(torch_cuda, closure):
    """Minerbo and Eddington closures: both radiation stages agree with the
    oracle to 1e-12 per cell (random fluxes, some |f| > 1), and 5 full RHD
    steps to 1e-10."""
    torch = torch_cuda
    lay = P.two_patches((11, 9, 7))
    U, R = _state_with_boundary(lay, (0, 0, 0), (0, 0, 0), seed=13)
    # a few superluminal states exercise the rescaling and the first-order fallback
    rng = np.random.Generator(np.random.Philox(2))
    for b in range(lay.nbox):
        hit = rng.random(lay.interior(R[1], b).shape) < 0.03
        for d in range(3):
            lay.interior(R[1 + d], b)[hit] *= 1.8
    prm = dict(PRM, closure=closure)
    g, p = _grid(lay), O.make_params(**prm)
    dtr = 0.3 * 0.1 / prm["chat"]
    for a in U + R:
        O.fill_ghosts(g, a)
    R1r = [np.zeros_like(a) for a in R]
    O.rad_stage(g, p, 1, R, None, R1r, U[0], dtr)
    R2r = [a.copy() for a in R]
    O.rad_stage(g, p, 2, R2r, R1r, R2r, U[0], dtr)
    ctx = _ctx(lay, prm)
    dR0, drho = G.dev(R), G.dev([U[0]])[0]
    dR1 = G.dev([np.zeros_like(a) for a in R])
    ctx.rad_stage(1, dR0, None, dR1, drho, dtr)
    e1 = G.max_rel_err(lay, G.host(dR1), R1r)
    dR1 = G.dev(R1r)
    ctx.fill_ghosts(dR1, 5)
    ctx.rad_stage(2, dR0, dR1, dR0, drho, dtr)
    torch.cuda.synchronize()
    e2 = G.max_rel_err(lay, G.host(dR0), R2r)
    ctx.close()
    assert max(e1) <= TOL_STAGE and max(e2) <= TOL_STAGE, (e1, e2)
    Ug, Rg, hg, st = _gpu_steps(lay, prm, U, R, 5)
    Ur, Rr, hr = _oracle_steps(lay, prm, U, R, 5)
    assert st[0] == 0
    _check_hist(hg, hr)
    e = G.max_rel_err(lay, Ug + Rg, Ur + Rr)
    assert max(e) <= TOL_STEPS, e


def test_source_matches_oracle(torch_cuda):
    """The emissivity field of the exchange (S = dt (chat/c) j): one exchange
    agrees with the oracle to 1e-12 per cell, 5 full steps to 1e-10; the
    FP32-mixed exchange with the source within 1e-5 relative L1."""
    torch = torch_cuda
    lay = P.two_patches((11, 9, 7))
    U, R = _state_with_boundary(lay, (0, 0, 0), (0, 0, 0), seed=14)
    rng = np.random.Generator(np.random.Philox(6))
    j = np.zeros(lay.field_len)
    for b in range(lay.nbox):
        lay.interior(j, b)[...] = 50.0 * rng.random(lay.interior(j, b).shape)
    prm = dict(PRM)
    g, p = _grid(lay), O.make_params(**prm)
    dtr = 0.3 * 0.1 / prm["chat"]
    Ur, Rr = [a.copy() for a in U], [a.copy() for a in R]
    rc, _ = O.exchange(g, p, Ur, Rr, dtr, src=j)
    assert rc == 0
    for prec in (0, 1):
        dt = torch.float64 if prec == 0 else torch.float32
        ctx = _ctx(lay, prm, prec)
        dU, dR = G.dev(U, dt), G.dev(R, dt)
        dj = G.dev([j], dt)[0]
        ctx.set_source(dj)
        ctx.exchange(dU, dR, dtr)
        torch.cuda.synchronize()
        assert ctx.status()[0] == 0
        if prec == 0:
            e = G.max_rel_err(lay, G.host(dU) + G.host(dR), Ur + Rr)
            assert max(e) <= TOL_STAGE, e
        else:
            l1 = G.rel_l1(lay, [G.host(dU)[4], G.host(dR)[0]], [Ur[4], Rr[0]])
            assert max(l1) <= 1e-5, l1
        ctx.close()
    Ug, Rg, hg, st = _gpu_steps(lay, prm, U, R, 5, src=j)
    Uo, Ro, ho = _oracle_steps(lay, prm, U, R, 5, src=j)
    assert st[0] == 0
    _check_hist(hg, ho)
    e = G.max_rel_err(lay, Ug + Rg, Uo + Ro)
    assert max(e) <= TOL_STEPS, e


def _tube():
    spec = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_values.json")))["radiation_pressure_tube"]
    return spec, P.radiation_pressure_tube(spec)


def _tube_temperatures(lay, U, R, prm):
    rho = lay.interior(U[0], 0).ravel()
    m = lay.interior(U[1], 0).ravel()
    Tg = (lay.interior(U[4], 0).ravel() - 0.5 * m * m / rho) / (rho * prm["c_v"])
    Tr = (lay.interior(R[0], 0).ravel() / prm["a_r"]) ** 0.25
    return Tg, Tr


def test_radiation_pressure_tube_gpu(torch_cuda):
    """Sec. 3.3.1 on the GPU through qk_step (Dirichlet states of all nine
    fields, tau_cell ~ 100): after one sound-crossing time the mean relative
    temperature error stays within the paper's 0.2 % and the final state
    agrees with the oracle's to 1e-9 per cell (FP64)."""
    torch = torch_cuda
    spec, (lay, U, R, prm, Tex, t_end) = _tube()
    ctx = _ctx(lay, prm)
    dU, dR = G.dev(U), G.dev(R)
    ctx.set_dirichlet(dU, dR)
    t, steps = 0.0, 0
    while t < t_end:
        dt, _ = ctx.step(dU, dR, want_dt=True)
        t += dt
        steps += 1
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0
    ctx.close()
    Ug, Rg = G.host(dU), G.host(dR)
    for T in _tube_temperatures(lay, Ug, Rg, prm):
        assert np.abs(T / Tex - 1).mean() < spec["rel_error"]
    Uo, Ro, _ = _oracle_steps(lay, prm, U, R, steps)
    e = G.max_rel_err(lay, Ug + Rg, Uo + Ro)
    assert max(e) <= 1e-9, e


def test_sharded_step_with_boundaries_bit_identical(torch_cuda):
    """Two virtual ranks with reflecting, outflow and Dirichlet faces (the
    sign flips travel in the packed halos; each rank restores its own
    Dirichlet states) give bit for bit the single-context qk_step."""
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    bc_lo, bc_hi = BCS["mixed_faces"]
    lay = I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=4, edges=(8, 16, 24))
    U, R = _state_with_boundary(lay, bc_lo, bc_hi, seed=15)
    prm = dict(PRM, bc_lo=bc_lo, bc_hi=bc_hi, dx=1.0 / 48)
    ref_U, ref_R, href, _ = _gpu_steps(lay, prm, U, R, 2)
    owner = S.partition(lay, 2)
    ranks = []
    for r in range(2):
        rlay = S.rank_layout(lay, owner, r)
        ctx = qk.Context(rlay, prm, 0, owner=owner, rank=r)
        fields = []
        for a in U + R:
            x = np.zeros(rlay.field_len)
            for b in np.nonzero(owner == r)[0]:
                rlay.full(x, b)[...] = lay.full(a, b)
            fields.append(x)
        d = G.dev(fields)
        ctx.set_dirichlet(d[:5], d[5:])
        ranks.append((rlay, ctx, S.RankStepper(ctx, d[:5], d[5:])))
    hist = [S.run_local([st for _, _, st in ranks])[0] for _ in range(2)]
    assert [(a, int(b)) for a, b in hist] == [(a, int(b)) for a, b in href]
    for r, (rlay, ctx, st) in enumerate(ranks):
        got = G.host(st.U) + G.host(st.R)
        for f in range(9):
            for b in np.nonzero(owner == r)[0]:
                assert np.array_equal(rlay.interior(got[f], b),
                                      lay.interior((ref_U + ref_R)[f], b))
        ctx.close()
