"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  FP64: max relative error per cell (floor = RMS of the
field) <= 1e-12 for one stage, <= 1e-10 after 10 steps; the ghost fill is
bit-exact.  FP32-mixed: relative L1 error <= 1e-5 in rho, E, E_r."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from tests import gpu_util as G
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL_STAGE = 1e-12
TOL_STEPS = 1e-10
TOL_MIXED_L1 = 1e-5
# FP32 stage against the FP64 oracle, per field (see _check_fp32_stage):
# 8 and 168 FP32 ulps (2^-24)
TOL_FP32_L1 = 8 * 2.0 ** -24
TOL_FP32_MAX = 168 * 2.0 ** -24


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


def _ctx(lay, prm, prec=0):
    from paper_2110_01792_gb300 import qk
    return qk.Context(lay, prm, prec)


def _grid(lay):
    return O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)


RAGGED = I.make_layout([[0, 0, 0], [13, 0, 0], [0, 7, 0]],
                       [[13, 7, 11], [6, 17, 11], [13, 10, 11]], (19, 17, 11), 4)


def _random_rhd(lay, seed, kappa0=None):
    prob = I.rhd_lognormal(layout=lay, seed=seed)
    # give the gas some velocity and the radiation some flux, incl. |f| > 1 spots
    rng = np.random.Generator(np.random.Philox(seed + 100))
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        v = 0.3 * rng.standard_normal((3,) + rho.shape)
        for d in range(3):
            lay.interior(prob.U[1 + d], b)[...] = rho * v[d]
        lay.interior(prob.U[4], b)[...] += 0.5 * rho * (v ** 2).sum(0)
        Er = lay.interior(prob.R[0], b)
        f = rng.standard_normal((3,) + Er.shape)
        f *= (0.9 * rng.random(Er.shape) / np.sqrt((f ** 2).sum(0)))
        f[:, rng.random(Er.shape) < 0.03] *= 1.3  # a few superluminal states
        for d in range(3):
            lay.interior(prob.R[1 + d], b)[...] = prob.params["c"] * Er * f[d]
    prm = dict(prob.params)
    prm["dx"] = 1.0 / max(lay.dom_n)
    if kappa0 is not None:
        prm["kappa_mode"] = 1
        prm["kappa_P"] = prm["kappa_R"] = kappa0
    return prob, prm


# ------------------------------------------------------------ ghost fill --

@pytest.mark.parametrize("prec", [0, 1])
def test_ghost_fill_bit_exact(torch_cuda, prec):
    torch = torch_cuda
    for lay in (I.single_box(13, 10, 9, ng=4), RAGGED,
                I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=3, edges=(8, 16, 24)),
                I.single_box(9, 1, 2, ng=4)):
        rng = np.random.Generator(np.random.Philox(1))
        fields = [rng.standard_normal(lay.field_len) for _ in range(9)]
        for f in fields:  # the interior only; the ghosts hold garbage
            pass
        ref = [f.copy() for f in fields]
        g = _grid(lay)
        for f in ref:
            O.fill_ghosts(g, f)
        ctx = _ctx(lay, dict(hydro_only=1, dx=0.1), prec)
        dt = torch.float64 if prec == 0 else torch.float32
        d = G.dev(fields, dt)
        ctx.fill_ghosts(d)
        torch.cuda.synchronize()
        for got, r in zip(G.host(d), ref):
            rr = r if prec == 0 else r.astype(np.float32).astype(np.float64)
            for b in range(lay.nbox):
                assert np.array_equal(lay.full(got, b), lay.full(rr, b))
        ctx.close()


# ----------------------------------------------------------- hydro stage --

@pytest.mark.parametrize("lay", [RAGGED, I.single_box(16, ng=4)], ids=["ragged", "box16"])
def test_hydro_stages_match_oracle(torch_cuda, lay):
    torch = torch_cuda
    prob, prm = _random_rhd(lay, 3)
    prm["hydro_only"] = 1
    U0 = prob.U
    p = O.make_params(**prm)
    g = _grid(lay)
    dt = 0.2 * O.timestep(g, p, U0)[0]
    U1r = [np.zeros_like(a) for a in U0]
    O.hydro_stage(g, p, 1, U0, None, U1r, dt)
    U2r = [a.copy() for a in U0]
    O.hydro_stage(g, p, 2, U2r, U1r, U2r, dt)
    ctx = _ctx(lay, prm)
    dU0 = G.dev(U0)
    dU1 = G.dev([np.zeros_like(a) for a in U0])
    ctx.fill_ghosts(dU0)
    ctx.hydro_stage(1, dU0, None, dU1, dt)
    e1 = G.max_rel_err(lay, G.host(dU1), U1r)
    # stage 2 from the oracle's U1 so that the two stages are checked separately
    dU1 = G.dev(U1r)
    ctx.fill_ghosts(dU1)
    ctx.hydro_stage(2, dU0, dU1, dU0, dt)
    torch.cuda.synchronize()
    e2 = G.max_rel_err(lay, G.host(dU0), U2r)
    ctx.close()
    assert max(e1) <= TOL_STAGE, e1
    assert max(e2) <= TOL_STAGE, e2


@pytest.mark.parametrize("shape", ["tiles", "columns"])
def test_hydro_stages_supersonic_match_oracle(torch_cuda, shape):
    """Every HLLC region on the GPU: a bulk flow at 3 times the reference
    sound speed in a random direction per patch (local Mach numbers from ~0.4
    to ~20: supersonic faces upwinding to either side, subsonic ones),
    converging and diverging neighbours across patch faces and velocity noise
    of 0.3 c_s (one, both or no side shocked in the PVRS estimate), density
    and pressure varying by e^4 from cell to cell; one stage each, FP64
    within 1e-12 of the oracle per cell, with the tile and the column
    kernels."""
    torch = torch_cuda
    lay = RAGGED
    prob, prm = _random_rhd(lay, 11)
    prm["hydro_only"] = 1
    rng = np.random.Generator(np.random.Philox(211))
    U0 = [a.copy() for a in prob.U]
    for b in range(lay.nbox):
        shp = lay.interior(U0[0], b).shape
        rho = np.exp(rng.uniform(-2.0, 2.0, shp))
        P = np.exp(rng.uniform(-2.0, 2.0, shp))
        cs = np.sqrt(prm["gamma"] * P / rho)
        d0 = rng.standard_normal(3)
        d0 /= np.linalg.norm(d0)
        v = (3.0 * math.sqrt(prm["gamma"]) * d0[:, None, None, None]
             + 0.3 * cs * rng.standard_normal((3,) + shp))
        lay.interior(U0[0], b)[...] = rho
        for d in range(3):
            lay.interior(U0[1 + d], b)[...] = rho * v[d]
        lay.interior(U0[4], b)[...] = P / (prm["gamma"] - 1.0) + 0.5 * rho * (v ** 2).sum(0)
    p = O.make_params(**prm)
    g = _grid(lay)
    dt = 0.2 * O.timestep(g, p, U0)[0]
    U1r = [np.zeros_like(a) for a in U0]
    O.hydro_stage(g, p, 1, U0, None, U1r, dt)
    U2r = [a.copy() for a in U0]
    O.hydro_stage(g, p, 2, U2r, U1r, U2r, dt)
    ctx = _ctx(lay, prm)
    if shape == "columns":
        ctx.set_launch_config(ALLCOLS)
    dU0 = G.dev(U0)
    dU1 = G.dev([np.zeros_like(a) for a in U0])
    ctx.fill_ghosts(dU0)
    ctx.hydro_stage(1, dU0, None, dU1, dt)
    e1 = G.max_rel_err(lay, G.host(dU1), U1r)
    dU1 = G.dev(U1r)
    ctx.fill_ghosts(dU1)
    ctx.hydro_stage(2, dU0, dU1, dU0, dt)
    torch.cuda.synchronize()
    e2 = G.max_rel_err(lay, G.host(dU0), U2r)
    ctx.close()
    assert max(e1) <= TOL_STAGE, e1
    assert max(e2) <= TOL_STAGE, e2


def _check_fp32_stage(lay, got, ref, tag):
    """One FP32 stage against the FP64 oracle's stage from the same inputs,
    per field: relative L1 and max relative error (RMS floor).  The FP32
    result carries the rounding of its FP32 inputs and output (half an ulp,
    2^-25, each), the approximate reciprocal / square root / quotient of the
    FP32 arithmetic (a few ulp) and their propagation through the stencil
    (the stage adds dt L, a fraction of the value, whose own relative error
    is that of a difference of face fluxes): a few ulps on average, relative
    L1 <= 8 ulp (4.8e-7; measured 0.7-1.7 ulp), and tens of ulps in the
    worst cell, max relative <= 168 ulp (1e-5; measured up to 18 ulp).  The
    max bound keeps room for a limiter decision of PPM or of the HLLC region
    taken at a near-tie, which FP32 may decide the other way than FP64."""
    l1 = G.rel_l1(lay, got, ref)
    mx = G.max_rel_err(lay, got, ref)
    print(f"fp32 vs oracle {tag}: rel_l1 max {max(l1):.3e} max_rel max {max(mx):.3e}")
    assert max(l1) <= TOL_FP32_L1, (tag, l1)
    assert max(mx) <= TOL_FP32_MAX, (tag, mx)


COLS = {"hydro1": (256, "columns"), "hydro2": (256, "columns"), "rad1": (256, "strided"),
        "rad2": (256, "strided")}


@pytest.mark.parametrize("recon,flat", [(0, 0), (1, 0), (0, 1)], ids=["ppm", "plm", "ppm_flat"])
@pytest.mark.parametrize("lay", [RAGGED, I.single_box(40, ng=4)], ids=["ragged", "box40"])
def test_column_hydro_stages_match_oracle(torch_cuda, lay, recon, flat):
    """The plane-marching form of the hydro stage (16 x 16 columns walking
    along z, partial footprints, z chunks): FP64 agrees with the oracle to
    1e-12 per stage; FP32 (columns and 8^3 tiles) agrees with the FP64
    oracle within the FP32 bounds of _check_fp32_stage."""
    torch = torch_cuda
    prob, prm = _random_rhd(lay, 4)
    prm["hydro_only"] = 1
    prm["recon"] = recon
    prm["flattening"] = flat
    U0 = prob.U
    p = O.make_params(**prm)
    g = _grid(lay)
    dt = 0.2 * O.timestep(g, p, U0)[0]
    U1r = [np.zeros_like(a) for a in U0]
    O.hydro_stage(g, p, 1, U0, None, U1r, dt)
    U2r = [a.copy() for a in U0]
    O.hydro_stage(g, p, 2, U2r, U1r, U2r, dt)
    for prec in (0, 1):
        tdt = torch.float64 if prec == 0 else torch.float32
        res = []
        for cfg in (COLS, None):
            ctx = _ctx(lay, prm, prec)
            if cfg is not None:
                ctx.set_launch_config(cfg)
            dU0 = G.dev(U0, tdt)
            dU1 = G.dev([np.zeros_like(a) for a in U0], tdt)
            ctx.fill_ghosts(dU0)
            ctx.hydro_stage(1, dU0, None, dU1, dt)
            s1 = G.host(dU1)
            dU1 = G.dev(U1r, tdt)
            ctx.fill_ghosts(dU1)
            ctx.hydro_stage(2, dU0, dU1, dU0, dt)
            torch.cuda.synchronize()
            res.append((s1, G.host(dU0)))
            ctx.close()
        (c1, c2), (t1, t2) = res
        if prec == 0:
            e1 = G.max_rel_err(lay, c1, U1r)
            e2 = G.max_rel_err(lay, c2, U2r)
            assert max(e1) <= TOL_STAGE and max(e2) <= TOL_STAGE, (e1, e2)
        else:
            for tag, a, ref in (("col1", c1, U1r), ("col2", c2, U2r), ("tile1", t1, U1r),
                                ("tile2", t2, U2r)):
                _check_fp32_stage(lay, a, ref, tag)


@pytest.mark.parametrize("lay", [RAGGED, I.single_box(40, ng=4)], ids=["ragged", "box40"])
def test_column_hydro_fp32_thread_counts_bit_identical(torch_cuda, lay):
    """The FP32 hydro column kernels with 288 threads per CTA (a ninth warp
    that owns no cell and takes x/y items and ring cells), registers held to 3
    or 2 CTAs per SM, compute every cell with the same arithmetic as the
    256-thread kernel: both stages bit-identical, partial footprints and z
    chunks included."""
    torch = torch_cuda
    prob, prm = _random_rhd(lay, 6)
    prm["hydro_only"] = 1
    p = O.make_params(**prm)
    dt = 0.2 * O.timestep(_grid(lay), p, prob.U)[0]
    res = []
    for cfg in ((256, "columns"), (288, "columns"), (288, "columns2")):
        ctx = _ctx(lay, prm, 1)
        ctx.set_launch_config({"hydro1": cfg, "hydro2": cfg, "rad1": (256, "strided"),
                               "rad2": (256, "strided")})
        dU0 = G.dev(prob.U, torch.float32)
        dU1 = G.dev([np.zeros_like(a) for a in prob.U], torch.float32)
        ctx.fill_ghosts(dU0)
        ctx.hydro_stage(1, dU0, None, dU1, dt)
        ctx.fill_ghosts(dU1)
        ctx.hydro_stage(2, dU0, dU1, dU0, dt)
        torch.cuda.synchronize()
        res.append(G.host(dU1) + G.host(dU0))
        ctx.close()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert np.array_equal(G.interior(lay, a), G.interior(lay, b))


@pytest.mark.parametrize("kappa0", [None, 60.0], ids=["thin", "thick_kappa_rho"])
@pytest.mark.parametrize("lay", [RAGGED, I.single_box(40, ng=4)], ids=["ragged", "box40"])
def test_column_rad_fp32_thread_counts_bit_identical(torch_cuda, lay, kappa0):
    """The FP32 Levermore radiation column kernels with 256 threads (the
    reconstruction positions past one per thread split by field across warps,
    the face pairs past one per thread solved as single faces on one warp)
    and with 288 threads (one pair per thread), registers held to 3 or 2 CTAs
    per SM: both stages and stage 2 with the exchange fused are
    bit-identical, superluminal fallbacks and the optical-depth correction
    included.  The random state drives a few cells of the thick case to
    negative energies in the exchange, which the status flags (equal in
    every configuration); their values are not defined and are left out of
    the comparison of the exchanged fields."""
    torch = torch_cuda
    prob, prm = _random_rhd(lay, 8, kappa0)
    dtr = 0.3 * (1.0 / max(lay.dom_n)) / prm["chat"]
    res = []
    for cfg in ((256, "columns"), (288, "columns"), (288, "columns2")):
        ctx = _ctx(lay, prm, 1)
        ctx.set_launch_config({"hydro1": (256, "strided"), "hydro2": (256, "strided"),
                               "rad1": cfg, "rad2": cfg})
        dR0 = G.dev(prob.R, torch.float32)
        dU = G.dev(prob.U, torch.float32)
        dR1 = G.dev([np.zeros_like(a) for a in prob.R], torch.float32)
        dR2 = G.dev([np.zeros_like(a) for a in prob.R], torch.float32)
        ctx.fill_ghosts(dR0 + [dU[0]])
        ctx.rad_stage(1, dR0, None, dR1, dU[0], dtr)
        ctx.fill_ghosts(dR1)
        ctx.rad_stage(2, dR0, dR1, dR2, dU[0], dtr)
        ctx.rad_stage2_exchange(dR0, dR1, dR0, dU, dtr)
        torch.cuda.synchronize()
        res.append(G.host(dR1) + G.host(dR2) + G.host(dR0) + G.host(dU) + [ctx.status()[1:]])
        ctx.close()
    names = ([f"R1[{q}]" for q in range(4)] + [f"R2[{q}]" for q in range(4)]
             + [f"R2x[{q}]" for q in range(4)] + [f"U[{q}]" for q in range(5)])
    # cells whose exchange ended with positive E_r and E in every configuration
    ok = np.ones(G.interior(lay, res[0][8]).shape, bool)
    for r in res:
        ok &= (G.interior(lay, r[8]) > 0) & (G.interior(lay, r[16]) > 0)
    if not ok.all():
        assert res[0][-1][0] & (1 << 4), res[0][-1]  # QK_ENEGATIVE raised
    assert ok.mean() > 0.99
    for k, other in enumerate(res[1:]):
        assert other[-1] == res[0][-1]  # exchange status: flags, first bad cell, iterations
        bad = []
        for j, (nm, a, b) in enumerate(zip(names, res[0][:-1], other[:-1])):
            ia, ib = G.interior(lay, a), G.interior(lay, b)
            if j >= 8:
                ia, ib = ia[ok], ib[ok]
            if not np.array_equal(ia, ib):
                i = int(np.argmax(np.abs(ia - ib)))
                bad.append((nm, int((ia != ib).sum()), i, float(ia[i]), float(ib[i])))
        assert not bad, (k + 1, bad)


def test_column_hydro_ten_steps_fp64(torch_cuda):
    """10 FP64 hydro steps of the seeded 32^3 workload with the column kernels
    agree with the oracle to 1e-10 per cell."""
    prob = I.config("hydro32")
    Ug, _, hg, st = _run_gpu_steps(prob.layout, prob, prob.params, 10, launch=COLS)
    Ur, _, hr = _run_oracle_steps(prob.layout, prob, prob.params, 10)
    _check_dt(hg, hr)
    e = G.max_rel_err(prob.layout, Ug, Ur)
    assert max(e) <= TOL_STEPS, e


# ------------------------------------------------------------- rad stage --

@pytest.mark.parametrize("kappa0", [None, 60.0], ids=["thin", "thick_kappa_rho"])
def test_rad_stages_match_oracle(torch_cuda, kappa0):
    torch = torch_cuda
    lay = RAGGED
    prob, prm = _random_rhd(lay, 4, kappa0)
    p = O.make_params(**prm)
    g = _grid(lay)
    dtr = 0.3 * (1.0 / 19) / prm["chat"]
    rho = prob.U[0]
    R1r = [np.zeros_like(a) for a in prob.R]
    O.rad_stage(g, p, 1, prob.R, None, R1r, rho, dtr)
    R2r = [a.copy() for a in prob.R]
    O.rad_stage(g, p, 2, R2r, R1r, R2r, rho, dtr)
    ctx = _ctx(lay, prm)
    dR0 = G.dev(prob.R)
    drho = G.dev([rho])[0]
    dR1 = G.dev([np.zeros_like(a) for a in prob.R])
    ctx.fill_ghosts(dR0 + [drho])
    ctx.rad_stage(1, dR0, None, dR1, drho, dtr)
    e1 = G.max_rel_err(lay, G.host(dR1), R1r)
    dR1 = G.dev(R1r)
    ctx.fill_ghosts(dR1)
    ctx.rad_stage(2, dR0, dR1, dR0, drho, dtr)
    torch.cuda.synchronize()
    e2 = G.max_rel_err(lay, G.host(dR0), R2r)
    ctx.close()
    assert max(e1) <= TOL_STAGE, e1
    assert max(e2) <= TOL_STAGE, e2


ALLCOLS = {k: (256, "columns") for k in ("hydro1", "hydro2", "rad1", "rad2")}


@pytest.mark.parametrize("closure", [0, 1, 2], ids=["levermore", "minerbo", "eddington"])
@pytest.mark.parametrize("kappa0", [None, 60.0], ids=["thin", "thick_kappa_rho"])
@pytest.mark.parametrize("lay", [RAGGED, I.single_box(40, ng=4)], ids=["ragged", "box40"])
def test_column_rad_stages_match_oracle(torch_cuda, lay, kappa0, closure):
    """The plane-marching form of the radiation stage (16 x 16 columns along
    z; partial footprints, z chunks, superluminal fallbacks, the optical-depth
    correction, the three closures): FP64 agrees with the oracle to 1e-12 per
    stage; FP32 (columns and 8^3 tiles) agrees with the FP64 oracle within
    the FP32 bounds of _check_fp32_stage."""
    torch = torch_cuda
    prob, prm = _random_rhd(lay, 4, kappa0)
    prm["closure"] = closure
    p = O.make_params(**prm)
    g = _grid(lay)
    dtr = 0.3 * (1.0 / max(lay.dom_n)) / prm["chat"]
    rho = prob.U[0]
    R1r = [np.zeros_like(a) for a in prob.R]
    O.rad_stage(g, p, 1, prob.R, None, R1r, rho, dtr)
    R2r = [a.copy() for a in prob.R]
    O.rad_stage(g, p, 2, R2r, R1r, R2r, rho, dtr)
    for prec in (0, 1):
        tdt = torch.float64 if prec == 0 else torch.float32
        res = []
        for cfg in (ALLCOLS, None):
            ctx = _ctx(lay, prm, prec)
            if cfg is not None:
                ctx.set_launch_config(cfg)
            dR0 = G.dev(prob.R, tdt)
            drho = G.dev([rho], tdt)[0]
            dR1 = G.dev([np.zeros_like(a) for a in prob.R], tdt)
            ctx.fill_ghosts(dR0 + [drho])
            ctx.rad_stage(1, dR0, None, dR1, drho, dtr)
            s1 = G.host(dR1)
            dR1 = G.dev(R1r, tdt)
            ctx.fill_ghosts(dR1)
            ctx.rad_stage(2, dR0, dR1, dR0, drho, dtr)
            torch.cuda.synchronize()
            res.append((s1, G.host(dR0)))
            ctx.close()
        (c1, c2), (t1, t2) = res
        if prec == 0:
            e1 = G.max_rel_err(lay, c1, R1r)
            e2 = G.max_rel_err(lay, c2, R2r)
            assert max(e1) <= TOL_STAGE and max(e2) <= TOL_STAGE, (e1, e2)
        else:
            for tag, a, ref in (("col1", c1, R1r), ("col2", c2, R2r), ("tile1", t1, R1r),
                                ("tile2", t2, R2r)):
                _check_fp32_stage(lay, a, ref, tag)


@pytest.mark.parametrize("kappa_mode", [0, 1], ids=["kconst", "krho"])
def test_column_rhd_ten_steps_fp64(torch_cuda, kappa_mode):
    """10 full FP64 RHD steps with every stage on columns (the exchange fused
    into the column form of radiation stage 2) agree with the oracle to 1e-10
    per cell, with dt and N_sub equal."""
    lay, prob, prm = _small_rhd(kappa_mode=kappa_mode, sigma=1.5 if kappa_mode else 1.0)
    Ug, Rg, hg, st = _run_gpu_steps(lay, prob, prm, 10, launch=ALLCOLS)
    Ur, Rr, hr = _run_oracle_steps(lay, prob, prm, 10)
    assert st[0] == 0, st
    _check_dt(hg, hr)
    e = G.max_rel_err(lay, Ug + Rg, Ur + Rr)
    assert max(e) <= TOL_STEPS, e


def test_column_mixed_rhd_error(torch_cuda):
    """FP32-mixed RHD with every stage on columns stays within the mixed
    bound (relative L1 <= 1e-5 in rho, E, E_r) of the FP64 oracle."""
    lay, prob, prm = _small_rhd()
    Ug, Rg, _, st = _run_gpu_steps(lay, prob, prm, 10, prec=1, launch=ALLCOLS)
    Ur, Rr, _ = _run_oracle_steps(lay, prob, prm, 10)
    assert st[0] == 0
    l1 = G.rel_l1(lay, [Ug[0], Ug[4], Rg[0]], [Ur[0], Ur[4], Rr[0]])
    assert max(l1) <= TOL_MIXED_L1, l1


# -------------------------------------------------------------- exchange --

@pytest.mark.parametrize("kappa0", [None, 40.0], ids=["kconst", "krho"])
def test_exchange_matches_oracle(torch_cuda, kappa0):
    torch = torch_cuda
    lay = RAGGED
    prob, prm = _random_rhd(lay, 5, kappa0)
    p = O.make_params(**prm)
    g = _grid(lay)
    dtr = 0.3 * (1.0 / 19) / prm["chat"]
    Ur = [a.copy() for a in prob.U]
    Rr = [a.copy() for a in prob.R]
    rc, info = O.exchange(g, p, Ur, Rr, dtr)
    assert rc == 0
    ctx = _ctx(lay, prm)
    dU, dR = G.dev(prob.U), G.dev(prob.R)
    ctx.exchange(dU, dR, dtr)
    torch.cuda.synchronize()
    rc, flags, bad, maxit = ctx.status()
    # the FP64 iteration starts from an FP32 Newton solve, so it takes at most
    # as many steps as the oracle's from the cell state (and at least the
    # correction plus the confirming step)
    assert rc == 0 and flags == 0 and bad == -1 and 2 <= maxit <= info[2] + 1, (maxit, info)
    e = G.max_rel_err(lay, G.host(dU) + G.host(dR), Ur + Rr)
    ctx.close()
    assert max(e) <= TOL_STAGE, e


def _cgs_state(lay, seed):
    """The random RHD state rescaled to cgs magnitudes (rho ~ 1e-2 g/cm^3,
    T ~ 1e7 K, c_v = 1.24e8, a_r = 7.56e-15, c = 3e10 cm/s, chat = 10 c_s:
    E_g ~ 1e13 and E_r ~ 1e14 erg/cm^3), with its parameters."""
    prob, prm = _random_rhd(lay, seed)
    gamma, c_v, T0, a_r, c = prm["gamma"], 1.24e8, 1e7, 7.56e-15, 3e10
    cs0 = math.sqrt(gamma * (gamma - 1.0) * c_v * T0)
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R]
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        v = [lay.interior(prob.U[1 + d], b) / rho for d in range(3)]
        Er = lay.interior(prob.R[0], b)
        f = [lay.interior(prob.R[1 + d], b) / (prm["c"] * Er) for d in range(3)]
        rho2 = 1e-2 * rho
        v2 = [cs0 * x for x in v]
        lay.interior(U[0], b)[...] = rho2
        for d in range(3):
            lay.interior(U[1 + d], b)[...] = rho2 * v2[d]
        lay.interior(U[4], b)[...] = rho2 * c_v * T0 + 0.5 * rho2 * sum(x * x for x in v2)
        Er2 = a_r * T0 ** 4 * Er  # E_r = T_r^4 in the code-unit state
        lay.interior(R[0], b)[...] = Er2
        for d in range(3):
            lay.interior(R[1 + d], b)[...] = c * Er2 * f[d]
    prm = dict(prm, c_v=c_v, a_r=a_r, c=c, chat=10.0 * cs0, kappa_P=1.0, kappa_R=1.0,
               kappa_mode=0)
    return U, R, prm


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_exchange_cgs_scales_matches_oracle(torch_cuda, prec):
    """The exchange on cgs-scaled states: E_g^4 overflows FP32 and
    A = k a_r/(rho c_v)^4 is not a normal float, so the FP32 warm start, the
    FP32-Jacobian and the double-float refinements stand aside and the full
    FP64 Newton iteration runs.  FP64 agrees with the oracle to 1e-12 per
    cell; FP32-mixed (FP32 state, oracle on the same rounded inputs) to the
    FP32 storage (4e-6) with no failure status."""
    torch = torch_cuda
    lay = RAGGED
    U, R, prm = _cgs_state(lay, 8)
    if prec == 1:
        U = [a.astype(np.float32).astype(np.float64) for a in U]
        R = [a.astype(np.float32).astype(np.float64) for a in R]
    dtr = 0.3 * (1.0 / 19) / prm["chat"]
    Ur = [a.copy() for a in U]
    Rr = [a.copy() for a in R]
    rc, info = O.exchange(_grid(lay), O.make_params(**prm), Ur, Rr, dtr)
    assert rc == 0
    ctx = _ctx(lay, prm, prec)
    tdt = torch.float64 if prec == 0 else torch.float32
    dU, dR = G.dev(U, tdt), G.dev(R, tdt)
    ctx.exchange(dU, dR, dtr)
    torch.cuda.synchronize()
    rc, flags, bad, maxit = ctx.status()
    ctx.close()
    assert rc == 0 and flags == 0 and bad == -1 and 1 <= maxit <= info[2] + 1, (maxit, info)
    e = G.max_rel_err(lay, G.host(dU) + G.host(dR), Ur + Rr)
    assert max(e) <= (TOL_STAGE if prec == 0 else 4e-6), e


@pytest.mark.parametrize("kappa_mode", [0, 1], ids=["kconst", "krho"])
def test_mixed_exchange_matches_oracle(torch_cuda, kappa_mode):
    """FP32-mixed exchange against the FP64 oracle on the same FP32-rounded
    state, with the opacity set so that k c/chat = dt rho kappa_P c (times rho
    for kappa = kappa0 rho) straddles the bound below which the refinement
    runs in double-float (k c/chat < eps 2^43 - 1, ~878 at eps = 1e-10):
    both the double-float and the FP64 refinement are exercised.  The FP32
    coefficients A, k and the FP32 storage bound the per-cell error
    (~1e-6 relative)."""
    torch = torch_cuda
    lay = RAGGED
    prob, prm = _random_rhd(lay, 7)
    rho = G.interior(lay, prob.U[0])
    dtr = 0.3 * (1.0 / 19) / prm["chat"]
    w = rho if kappa_mode == 0 else rho * rho
    prm["kappa_mode"] = kappa_mode
    prm["kappa_P"] = prm["kappa_R"] = 878.0 / (dtr * float(np.median(w)) * prm["c"])
    kcr = dtr * w * prm["kappa_P"] * prm["c"]
    assert 0.3 < np.mean(kcr < 850.0) < 0.7 and np.mean(kcr > 900.0) > 0.3
    U32 = [a.astype(np.float32).astype(np.float64) for a in prob.U]
    R32 = [a.astype(np.float32).astype(np.float64) for a in prob.R]
    Ur = [a.copy() for a in U32]
    Rr = [a.copy() for a in R32]
    rc, info = O.exchange(_grid(lay), O.make_params(**prm), Ur, Rr, dtr)
    assert rc == 0
    ctx = _ctx(lay, prm, 1)
    dU, dR = G.dev(U32, torch.float32), G.dev(R32, torch.float32)
    ctx.exchange(dU, dR, dtr)
    torch.cuda.synchronize()
    rc, flags, bad, maxit = ctx.status()
    ctx.close()
    assert rc == 0 and flags == 0 and bad == -1 and maxit <= info[2] + 1, (maxit, info)
    e = G.max_rel_err(lay, G.host(dU) + G.host(dR), Ur + Rr)
    assert max(e) <= 4e-6, e


def test_exchange_nonconvergence_reported(torch_cuda):
    torch = torch_cuda
    lay = I.single_box(3, 2, 2)
    prob = I.rhd_lognormal(layout=lay, seed=1)
    prm = dict(prob.params, max_iter=1, dx=1.0 / 3)
    ctx = _ctx(lay, prm)
    dU, dR = G.dev(prob.U), G.dev(prob.R)
    ctx.exchange(dU, dR, 0.5)
    torch.cuda.synchronize()
    from paper_2110_01792_gb300 import qk
    rc, flags, bad, maxit = ctx.status(reset=True)
    assert rc == qk.ENOCONV and flags & (1 << qk.ENOCONV)
    assert bad == int(lay.off[0]) + (4 * 10 + 4) * 11 + 4  # first interior cell
    rc2, flags2, bad2, _ = ctx.status()
    assert rc2 == 0 and flags2 == 0 and bad2 == -1
    ctx.close()


# ------------------------------------------------------- timestep, sums ---

@pytest.mark.parametrize("prec", [0, 1])
def test_timestep_matches_oracle(torch_cuda, prec):
    """dt, N_sub and dt_rad from the device reduction agree with the oracle
    (FP64: to a few ulp; FP32 state: to FP32 accuracy); N_sub exactly."""
    torch = torch_cuda
    lay = RAGGED
    prob, prm = _random_rhd(lay, 6)
    U = prob.U if prec == 0 else [a.astype(np.float32).astype(np.float64) for a in prob.U]
    p = O.make_params(**prm)
    ref = O.timestep(_grid(lay), p, U)
    smax = O.max_signal_speed(_grid(lay), p, U)
    ctx = _ctx(lay, prm, prec)
    got = ctx.timestep(G.dev(U, torch.float64 if prec == 0 else torch.float32))
    ctx.close()
    tol = 1e-14 if prec == 0 else 1e-6
    assert abs(got[3] - smax) <= tol * smax and abs(got[0] - ref[0]) <= tol * ref[0]
    assert got[1] == ref[1] and abs(got[2] - ref[2]) <= tol * ref[2]


def test_conserved_sums_match_oracle(torch_cuda):
    lay = RAGGED
    prob, prm = _random_rhd(lay, 7)
    ref = O.conserved_sums(_grid(lay), O.make_params(**prm), prob.U, prob.R)
    ctx = _ctx(lay, prm)
    got = ctx.conserved_sums(G.dev(prob.U), G.dev(prob.R))
    again = ctx.conserved_sums(G.dev(prob.U), G.dev(prob.R))
    ctx.close()
    assert np.array_equal(got, again)  # fixed reduction order
    for a, b in zip(got, ref):
        assert abs(a - b) <= 4e-16 * max(abs(b), 1e-300) + 1e-300


# --------------------------------------------------------- whole steps ----

def _run_gpu_steps(lay, prob, prm, nsteps, prec=0, graph=True, launch=None):
    torch = pytest.importorskip("torch")
    ctx = _ctx(lay, prm, prec)
    ctx.set_graph(graph)
    if launch is not None:
        ctx.set_launch_config(launch)
    dt_ = torch.float64 if prec == 0 else torch.float32
    dU = G.dev(prob.U, dt_)
    dR = G.dev(prob.R, dt_) if prob.R is not None else None
    hist = []
    for _ in range(nsteps):
        hist.append(ctx.step(dU, dR, want_dt=True))
    torch.cuda.synchronize()
    st = ctx.status()
    ctx.close()
    return G.host(dU), (G.host(dR) if dR is not None else None), hist, st


def _run_oracle_steps(lay, prob, prm, nsteps):
    g = _grid(lay)
    p = O.make_params(**prm)
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R] if prob.R is not None else None
    hist = []
    for _ in range(nsteps):
        rc, ts, info = O.step(g, p, U, R)
        assert rc == 0
        hist.append((ts[0], ts[1]))
    return U, R, hist


def test_hydro32_ten_steps_fp64(torch_cuda):
    """The hydro workload (32^3, seeded waves, PPM + HLLC + RK2, CFL 0.3):
    10 FP64 steps agree with the oracle to 1e-10 per cell, step sizes equal."""
    prob = I.config("hydro32")
    Ug, _, hg, st = _run_gpu_steps(prob.layout, prob, prob.params, 10)
    Ur, _, hr, = _run_oracle_steps(prob.layout, prob, prob.params, 10)[0:3]
    _check_dt(hg, hr)
    e = G.max_rel_err(prob.layout, Ug, Ur)
    assert max(e) <= TOL_STEPS, e


def _check_dt(hg, hr):
    """Step sizes agree to round-off (the states differ by round-off only);
    N_sub must agree."""
    for (dg, ng), (dr, nr) in zip(hg, hr):
        assert abs(dg - dr) <= 1e-13 * dr and int(ng) == int(nr)


def _small_rhd(kappa_mode=0, sigma=1.0):
    lay = I.make_layout([[0, 0, 0], [8, 0, 0], [0, 8, 0]], [[8, 8, 12], [12, 16, 12], [8, 8, 12]],
                        (20, 16, 12), 4)
    prob = I.rhd_lognormal(layout=lay, seed=9, sigma=sigma, kappa_mode=kappa_mode,
                           kappa0=1.0 if kappa_mode == 0 else 30.0)
    prm = dict(prob.params)
    prm["dx"] = 1.0 / 20
    return lay, prob, prm


@pytest.mark.parametrize("graph", [True, False])
def test_rhd_patches_ten_steps_fp64(torch_cuda, graph):
    """RHD on a 3-patch periodic set with ragged tiles: 10 full steps (hydro +
    N_sub radiation substeps + exchange) agree with the oracle to 1e-10 per
    cell; dt and N_sub agree exactly; no Newton failure."""
    lay, prob, prm = _small_rhd()
    Ug, Rg, hg, st = _run_gpu_steps(lay, prob, prm, 10, graph=graph)
    Ur, Rr, hr = _run_oracle_steps(lay, prob, prm, 10)
    assert st[0] == 0, st
    _check_dt(hg, hr)
    e = G.max_rel_err(lay, Ug + Rg, Ur + Rr)
    assert max(e) <= TOL_STEPS, e


def test_rhd_kappa_rho_ten_steps_fp64(torch_cuda):
    """kappa = kappa0 rho with optically thick cells (the optical-depth
    correction active) and sigma_ln rho = 1.5."""
    lay, prob, prm = _small_rhd(kappa_mode=1, sigma=1.5)
    Ug, Rg, hg, st = _run_gpu_steps(lay, prob, prm, 10)
    Ur, Rr, hr = _run_oracle_steps(lay, prob, prm, 10)
    assert st[0] == 0, st
    e = G.max_rel_err(lay, Ug + Rg, Ur + Rr)
    assert max(e) <= TOL_STEPS, e


def test_mixed_precision_error_bounds(torch_cuda):
    """FP32 state and stencils with FP64 Newton / E_g / sums: relative L1 error
    in rho, E and E_r against the FP64 oracle <= 1e-5 after 10 steps."""
    prob = I.config("hydro32")
    Ug, _, _, _ = _run_gpu_steps(prob.layout, prob, prob.params, 10, prec=1)
    Ur, _, _ = _run_oracle_steps(prob.layout, prob, prob.params, 10)
    l1 = G.rel_l1(prob.layout, [Ug[0], Ug[4]], [Ur[0], Ur[4]])
    assert max(l1) <= TOL_MIXED_L1, l1
    lay, prob, prm = _small_rhd()
    Ug, Rg, _, st = _run_gpu_steps(lay, prob, prm, 10, prec=1)
    Ur, Rr, _ = _run_oracle_steps(lay, prob, prm, 10)
    assert st[0] == 0
    l1 = G.rel_l1(lay, [Ug[0], Ug[4], Rg[0]], [Ur[0], Ur[4], Rr[0]])
    assert max(l1) <= TOL_MIXED_L1, l1


def test_stationary_contact_and_uniform_exact_on_gpu(torch_cuda):
    """Sec. 3.1.2 on the GPU: the stationary contact stays exactly unchanged
    (and so does a uniform moving state), in 3-D and through qk_step."""
    torch = torch_cuda
    N = 24
    lay = I.single_box(N, 8, 8, ng=4)
    U = I.zeros(lay, 5)
    x = P.centres(N)
    rho = np.where(x < 0.5, 1.4, 1.0)
    lay.interior(U[0], 0)[...] = rho[None, None, :]
    lay.interior(U[4], 0)[...] = 1.0 / 0.4
    prob = I.Problem("contact", lay, dict(gamma=1.4, cfl=0.3, dx=1.0 / N, hydro_only=1), U)
    Ug, _, _, _ = _run_gpu_steps(lay, prob, prob.params, 20)
    for a, b in zip(Ug, U):
        assert np.array_equal(G.interior(lay, a), G.interior(lay, b))


def test_step_conserves_on_gpu(torch_cuda):
    """Periodic FP64 RHD: sum rho exact to round-off, sum(E + (c/chat) E_r) and
    sum(m + F/(c chat)) to round-off, measured with qk_conserved_sums."""
    torch = torch_cuda
    lay, prob, prm = _small_rhd()
    ctx = _ctx(lay, prm)
    dU, dR = G.dev(prob.U), G.dev(prob.R)
    s0 = ctx.conserved_sums(dU, dR)
    for _ in range(5):
        ctx.step(dU, dR)
    s1 = ctx.conserved_sums(dU, dR)
    ctx.close()
    assert abs(s1[0] - s0[0]) <= 1e-14 * abs(s0[0])
    assert abs(s1[9] - s0[9]) <= 1e-13 * abs(s0[9])
    for d in range(3):
        assert abs(s1[10 + d] - s0[10 + d]) <= 1e-13 * abs(s0[9]) / 100.0


@pytest.mark.parametrize("shape", ["tiles", "columns"])
def test_per_patch_launches_match_batched(torch_cuda, shape):
    """One launch per patch and stage gives bit-identical results to the
    batched persistent launch over all patches (each tile's or column's
    arithmetic does not depend on which CTA runs it), with either tile shape."""
    lay, prob, prm = _small_rhd()
    outs = []
    for per_patch in (False, True):
        ctx = _ctx(lay, prm)
        if shape == "columns":
            ctx.set_launch_config(ALLCOLS)
        ctx.set_launch_mode(per_patch)
        dU, dR = G.dev(prob.U), G.dev(prob.R)
        for _ in range(3):
            ctx.step(dU, dR)
        outs.append(G.host(dU) + G.host(dR))
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(G.interior(lay, a), G.interior(lay, b))


@pytest.mark.parametrize("prec", [0, 1])
def test_fused_exchange_matches_separate_launch(torch_cuda, prec):
    """The exchange fused into the epilogue of radiation stage 2 gives the same
    bits as its own launch after the stage (it reads the same values), with a
    radiation source, in FP64 and FP32-mixed, and for a compensated state."""
    torch = torch_cuda
    lay, prob, prm = _small_rhd()
    tdt = torch.float64 if prec == 0 else torch.float32
    rng = np.random.Generator(np.random.Philox(5))
    src = rng.uniform(0.0, 2.0, lay.field_len)
    outs = []
    for fused in (True, False):
        for comp in ((False, True) if prec == 1 else (False,)):
            ctx = _ctx(lay, prm, prec)
            ctx.set_fused_exchange(fused)
            j = torch.from_numpy(src).to(tdt).cuda()
            ctx.set_source(j)
            dU, dR = G.dev(prob.U, tdt), G.dev(prob.R, tdt)
            lo = None
            if comp:
                lo = ([torch.zeros_like(a) for a in dU], [torch.zeros_like(a) for a in dR])
            for _ in range(3):
                ctx.step(dU, dR, lo=lo)
            st = ctx.status()
            ctx.close()
            assert st[0] == 0, st
            res = G.host(dU) + G.host(dR) + (G.host(lo[0]) + G.host(lo[1]) if comp else [])
            outs.append([G.interior(lay, a) for a in res])
    half = len(outs) // 2
    for a, b in zip(outs[:half], outs[half:]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_autotune_keeps_state_and_results(torch_cuda):
    """qk_autotune leaves the interior state untouched, returns one of the
    candidate configurations per stage kernel, and updates computed with the
    tuned configurations are bit-identical to the default ones."""
    lay, prob, prm = _small_rhd()
    outs = []
    for tune in (False, True):
        ctx = _ctx(lay, prm)
        dU, dR = G.dev(prob.U), G.dev(prob.R)
        if tune:
            before = G.host(dU) + G.host(dR)
            cfg = ctx.autotune(dU, dR)
            assert set(cfg) == {"hydro1", "hydro2", "rad1", "rad2"}
            for th, sch in cfg.values():
                assert th in (128, 256, 288, 512) and sch in ("strided", "contiguous", "columns",
                                                               "columns2")
            for a, b in zip(G.host(dU) + G.host(dR), before):
                assert np.array_equal(G.interior(lay, a), G.interior(lay, b))
        for _ in range(2):
            ctx.step(dU, dR)
        outs.append(G.host(dU) + G.host(dR))
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(G.interior(lay, a), G.interior(lay, b))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shock_tube_thin_axes_gpu(torch_cuda, axis):
    """A 1-D stationary shock tube (Sec. 3.1.3 states, 10/100 | 1/1) on an
    N x 1 x 1 periodic grid along each axis: 1-cell-thick axes wrap their ghost
    layers several times, and the strong discontinuities exercise every HLLC
    region and limiter branch; 20 steps agree with the oracle to 1e-10."""
    N = 64
    x = P.centres(N, 10.0)
    inside = (x >= 2.0) & (x < 8.0)
    lay, U = P.hydro_line(N, np.where(inside, 1.0, 10.0), np.where(inside, 0.3, -0.2),
                          np.where(inside, 1.0, 100.0), 1.4, axis=axis)
    dx = [1.0, 1.0, 1.0]
    dx[axis] = 10.0 / N
    prm = dict(gamma=1.4, cfl=0.3, dx=dx, hydro_only=1)
    prob = I.Problem("tube", lay, prm, U)
    Ug, _, hg, _ = _run_gpu_steps(lay, prob, prm, 20)
    Ur, _, hr = _run_oracle_steps(lay, prob, prm, 20)
    _check_dt(hg, hr)
    e = G.max_rel_err(lay, Ug, Ur)
    assert max(e) <= TOL_STEPS, e


@pytest.mark.parametrize("recon,flat", [(1, 0), (0, 1), (1, 1)], ids=["plm", "ppm_flat", "plm_flat"])
def test_stages_with_plm_and_flattening(torch_cuda, recon, flat):
    """PLM-MC reconstruction and Miller & Colella shock flattening (Sec. 2.2.1)
    on random data with strong compressive jumps: one hydro stage and one
    radiation stage (PLM for radiation too, never flattened) agree with the
    oracle to 1e-12."""
    torch = torch_cuda
    lay = RAGGED
    prob, prm = _random_rhd(lay, 8)
    rng = np.random.Generator(np.random.Philox(31))
    for b in range(lay.nbox):  # pressure jumps of a factor 2-10 with converging flow
        E = lay.interior(prob.U[4], b)
        E *= np.where(rng.random(E.shape) < 0.15, rng.uniform(2, 10, E.shape), 1.0)
    prm = dict(prm, recon=recon, flattening=flat)
    p = O.make_params(**prm)
    g = _grid(lay)
    dt = 0.2 * O.timestep(g, p, prob.U)[0]
    U1r = [np.zeros_like(a) for a in prob.U]
    O.hydro_stage(g, p, 1, prob.U, None, U1r, dt)
    dtr = 0.3 * (1.0 / 19) / prm["chat"]
    R1r = [np.zeros_like(a) for a in prob.R]
    O.rad_stage(g, p, 1, prob.R, None, R1r, prob.U[0], dtr)
    ctx = _ctx(lay, prm)
    dU, dR = G.dev(prob.U), G.dev(prob.R)
    dU1 = [torch.zeros_like(a) for a in dU]
    dR1 = [torch.zeros_like(a) for a in dR]
    ctx.fill_ghosts(dU + dR)
    ctx.hydro_stage(1, dU, None, dU1, dt)
    ctx.rad_stage(1, dR, None, dR1, dU[0], dtr)
    torch.cuda.synchronize()
    eh = G.max_rel_err(lay, G.host(dU1), U1r)
    er = G.max_rel_err(lay, G.host(dR1), R1r)
    ctx.close()
    assert max(eh) <= TOL_STAGE, eh
    assert max(er) <= TOL_STAGE, er


def test_shock_tube_with_flattening_ten_steps_gpu(torch_cuda):
    """The stationary shock tube of Sec. 3.1.3 (x0 = 2, rho/p = 10/100 | 1/1,
    CFL 0.1) with flattening: 40 steps on the GPU agree with the oracle to
    1e-10."""
    N = 200
    x = P.centres(N, 10.0)
    inside = (x >= 2.0) & (x < 8.0)
    lay, U = P.hydro_line(N, np.where(inside, 1.0, 10.0), 0.0, np.where(inside, 1.0, 100.0), 1.4)
    prm = dict(gamma=1.4, cfl=0.1, dx=[10.0 / N, 1.0, 1.0], hydro_only=1, flattening=1)
    prob = I.Problem("tube", lay, prm, U)
    Ug, _, hg, _ = _run_gpu_steps(lay, prob, prm, 40)
    Ur, _, hr = _run_oracle_steps(lay, prob, prm, 40)
    _check_dt(hg, hr)
    e = G.max_rel_err(lay, Ug, Ur)
    assert max(e) <= TOL_STEPS, e


def test_step_host_matches_device_step(torch_cuda):
    """qk_step_host (state in host memory: pinned tensors and pageable numpy
    arrays) gives bit for bit the device qk_step of the same state, FP64 and
    FP32-mixed, with the step size and N_sub reported alike."""
    torch = torch_cuda
    lay, prob, prm = _small_rhd()
    for prec in (0, 1):
        tdt = torch.float64 if prec == 0 else torch.float32
        ndt = np.float64 if prec == 0 else np.float32
        ctx = _ctx(lay, prm, prec)
        dU, dR = G.dev(prob.U, tdt), G.dev(prob.R, tdt)
        pU = [torch.from_numpy(a).to(tdt).pin_memory() for a in prob.U]
        pR = [torch.from_numpy(a).to(tdt).pin_memory() for a in prob.R]
        nU = [np.ascontiguousarray(a, dtype=ndt) for a in prob.U]
        nR = [np.ascontiguousarray(a, dtype=ndt) for a in prob.R]
        for _ in range(3):
            a = ctx.step(dU, dR, want_dt=True)
            b = ctx.step_host(pU, pR, want_dt=True)
            c = ctx.step_host(nU, nR, want_dt=True)
            assert a == b == c, (a, b, c)
        torch.cuda.synchronize()
        assert ctx.status()[0] == 0
        ctx.close()
        for d, p_, n_ in zip(G.host(dU) + G.host(dR), pU + pR, nU + nR):
            assert np.array_equal(G.interior(lay, d), G.interior(lay, p_.double().numpy()))
            assert np.array_equal(G.interior(lay, d), G.interior(lay, n_.astype(np.float64)))
