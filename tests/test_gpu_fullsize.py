"""Full-size parity on sampled cells: one hydro stage, one radiation stage and
one exchange of the benchmark workloads (128^3 RHD FP64, the ~1500-patch
tiling FP64, 512^3 RHD FP32-mixed), launched exactly as qk_step launches them,
against the oracle evaluated cell by cell on a sample (random interior cells
plus patch corners, tile edges and ragged edges) of the same input state."""
import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _sample(lay, n_random, seed=0):
    rng = np.random.Generator(np.random.Philox(seed))
    cells = []
    boxes = rng.integers(0, lay.nbox, size=n_random)
    for b in boxes:
        n = lay.n[b]
        cells.append([b, rng.integers(0, n[0]), rng.integers(0, n[1]), rng.integers(0, n[2])])
    for b in rng.integers(0, lay.nbox, size=min(lay.nbox, 24)):
        n = lay.n[b]
        for i in (0, n[0] - 1, min(7, n[0] - 1), min(8, n[0] - 1)):
            for j in (0, n[1] - 1):
                for k in (0, n[2] - 1):
                    cells.append([b, i, j, k])
    # unique cells: the in-place exchange must see each cell once
    return np.unique(np.array(cells, dtype=np.int32), axis=0)


def _elems(lay, cells):
    g = lay.ng
    out = []
    for b, i, j, k in cells:
        n = lay.n[b]
        sx, sy = n[0] + 2 * g, n[1] + 2 * g
        out.append(lay.off[b] + ((k + g) * sy + (j + g)) * sx + (i + g))
    return np.array(out, dtype=np.int64)


def _cmp(torch, got_dev, ref_host, el, fp64):
    idx = torch.from_numpy(el).cuda()
    worst = []
    for d, r in zip(got_dev, ref_host):
        gv = d[idx].double().cpu().numpy()
        rv = r[el]
        if fp64:
            floor = max(float(np.sqrt(np.mean(rv ** 2))), 1e-300)
            worst.append(float(np.max(np.abs(gv - rv) / np.maximum(np.abs(rv), floor))))
        else:
            worst.append(float(np.abs(gv - rv).sum() / max(np.abs(rv).sum(), 1e-300)))
    return worst


@pytest.mark.parametrize("name", ["rhd128", "patches", "rhd512_fp32"])
def test_fullsize_sampled_stages(torch_cuda, name):
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    if name == "rhd128":
        prob, prec = I.rhd_lognormal(128), qk.FP64
    elif name == "patches":
        prob, prec = I.rhd_lognormal(layout=I.patch_tiling()), qk.FP64
    else:
        prob, prec = I.rhd_lognormal(512, sigma=1.5, kappa_mode=1), qk.FP32_MIXED
    lay = prob.layout
    fp64 = prec == qk.FP64
    tdt = torch.float64 if fp64 else torch.float32
    # give the state velocity and flux so that every branch is exercised
    rng = np.random.Generator(np.random.Philox(7))
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        v = 0.2 * rng.standard_normal((3,) + rho.shape)
        for d in range(3):
            lay.interior(prob.U[1 + d], b)[...] = rho * v[d]
        lay.interior(prob.U[4], b)[...] += 0.5 * rho * (v ** 2).sum(0)
        Er = lay.interior(prob.R[0], b)
        for d in range(3):
            lay.interior(prob.R[1 + d], b)[...] = 30.0 * Er * rng.uniform(-1, 1, Er.shape) / 3
    U = prob.U if fp64 else [a.astype(np.float32).astype(np.float64) for a in prob.U]
    R = prob.R if fp64 else [a.astype(np.float32).astype(np.float64) for a in prob.R]
    del prob.U, prob.R
    ctx = qk.Context(lay, prob.params, prec)
    dU = [torch.from_numpy(a).to(tdt).cuda() for a in U]
    dR = [torch.from_numpy(a).to(tdt).cuda() for a in R]
    ctx.fill_ghosts(dU + dR)
    dt, nsub, dtr, smax = ctx.timestep(dU)
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    p = O.make_params(**prob.params)
    cells = _sample(lay, 400 if lay.nbox == 1 else 600)
    el = _elems(lay, cells)
    tol = 1e-12 if fp64 else 1e-5
    # hydro stage 1
    dU1 = [torch.empty_like(a) for a in dU]
    ctx.hydro_stage(1, dU, None, dU1, dt)
    ref = [np.empty_like(a) for a in U]
    O.hydro_stage(g, p, 1, U, None, ref, dt, cells=cells)
    e = _cmp(torch, dU1, ref, el, fp64)
    assert max(e) <= tol, ("hydro", e)
    del dU1
    # radiation stage 1
    dR1 = [torch.empty_like(a) for a in dR]
    ctx.rad_stage(1, dR, None, dR1, dU[0], dtr)
    refr = [np.empty_like(a) for a in R]
    O.rad_stage(g, p, 1, R, None, refr, U[0], dtr, cells=cells)
    e = _cmp(torch, dR1, refr, el, fp64)
    assert max(e) <= tol, ("rad", e)
    del dR1, refr, ref
    # exchange (in place on both sides)
    ctx.exchange(dU, dR, dtr)
    rc, info = O.exchange(g, p, U, R, dtr, cells=cells)
    assert rc == 0
    st = ctx.status()
    assert st[0] == qk.OK, st
    e = _cmp(torch, dU + dR, U + R, el, fp64)
    assert max(e) <= tol, ("exchange", e)
    ctx.close()
