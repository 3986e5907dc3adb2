"""Compensated FP32 state (qk_step_compensated): every conserved field held as
hi + lo.  Against the FP64 oracle it meets the FP32-mixed bound (relative L1
<= 1e-5 in every field), and the periodic conserved totals -- sum rho, sum m,
sum (E + (c/chat) E_r), sum (m + F/(c chat)) -- stay constant over 10 steps,
where plain FP32 storage drifts by rounding at ~1e-11 per step: to 1e-13 of
their magnitude with FP32 low parts (~48-bit values), and to the 1e-12 bound
of the mixed form with 16-bit low parts (QK_LO_I16, ~39-bit values, 6 bytes
per value)."""
import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL_L1 = 1e-5
TOL_DRIFT = {"f32": 1e-13, "i16": 1e-12}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _small_rhd():
    lay = I.make_layout([[0, 0, 0], [8, 0, 0], [0, 8, 0]], [[8, 8, 12], [12, 16, 12], [8, 8, 12]],
                        (20, 16, 12), 4)
    prob = I.rhd_lognormal(layout=lay, seed=9)
    # some gas velocity and radiation flux, so that every field moves
    rng = np.random.Generator(np.random.Philox(77))
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        v = 0.2 * rng.standard_normal((3,) + rho.shape)
        for d in range(3):
            lay.interior(prob.U[1 + d], b)[...] = rho * v[d]
        lay.interior(prob.U[4], b)[...] += 0.5 * rho * (v ** 2).sum(0)
        Er = lay.interior(prob.R[0], b)
        f = 0.3 * rng.standard_normal((3,) + Er.shape)
        for d in range(3):
            lay.interior(prob.R[1 + d], b)[...] = prob.params["c"] * Er * np.clip(f[d], -0.5, 0.5)
    prm = dict(prob.params)
    prm["dx"] = 1.0 / 20
    return lay, prob, prm


def _oracle(lay, prob, prm, nsteps):
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    p = O.make_params(**prm)
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R] if prob.R is not None else None
    for _ in range(nsteps):
        rc, _, _ = O.step(g, p, U, R)
        assert rc == 0
    return U, R


def _magnitudes(lay, U, R, cr, icc):
    """Per total: the scale its drift is measured against (sum of |terms|)."""
    def s(a):
        return float(np.abs(G.interior(lay, a)).sum())
    mom = [s(U[1 + d]) + (s(R[1 + d]) * icc if R is not None else 0.0) for d in range(3)]
    etot = s(U[4]) + (cr * s(R[0]) if R is not None else 0.0)
    return s(U[0]), mom, etot


def _lo_parts(torch, qk, arrays, fmt):
    """Device low parts of a state given in FP64: the FP32 rounding residual,
    as floats (f32) or in the 16-bit encoding (i16)."""
    out = []
    for a in arrays:
        hi = a.astype(np.float32)
        res = a - hi.astype(np.float64)
        if fmt == "i16":
            out.append(torch.from_numpy(qk.lo16_encode(hi, res)).cuda())
        else:
            out.append(torch.from_numpy(res).float().cuda())
    return out


def _run(torch, lay, prob, prm, nsteps, compensated):
    """compensated: False (plain FP32 storage), "f32" or "i16" low parts."""
    from paper_2110_01792_gb300 import qk
    ctx = qk.Context(lay, prm, qk.FP32_MIXED)
    if compensated == "i16":
        ctx.set_lo_format(qk.LO_I16)
    U = G.dev(prob.U, torch.float32)
    R = G.dev(prob.R, torch.float32) if prob.R is not None else None
    lo = None
    if compensated:
        # the FP32 rounding residual of the initial state is its low part
        lo = (_lo_parts(torch, qk, prob.U, compensated),
              _lo_parts(torch, qk, prob.R, compensated) if R is not None else None)
    sums = [ctx.conserved_sums(U, R, lo=lo)]
    for _ in range(nsteps):
        ctx.step(U, R, lo=lo)
        sums.append(ctx.conserved_sums(U, R, lo=lo))
    st = ctx.status()
    ctx.close()
    out = G.host(U) + (G.host(R) if R is not None else [])
    if compensated:
        los = lo[0] + (lo[1] if R is not None else [])
        if compensated == "i16":
            extra = [qk.lo16_decode(h.astype(np.float32), l.cpu().numpy())
                     for h, l in zip(out, los)]
        else:
            extra = G.host(los)
        out = [a + b for a, b in zip(out, extra)]
    return out, np.array(sums), st


def _drift(sums, mags):
    rho_m, mom_m, etot_m = mags
    d = np.abs(sums - sums[0])
    return {"rho": d[:, 0].max() / rho_m,
            "E_total": d[:, 9].max() / etot_m,
            "momentum": max(d[:, 10 + a].max() / mom_m[a] for a in range(3))}


@pytest.mark.parametrize("fmt", ["f32", "i16"])
def test_compensated_hydro_accuracy_and_conservation(torch_cuda, fmt):
    prob = I.config("hydro32")
    lay, prm = prob.layout, prob.params
    got, sums, st = _run(torch_cuda, lay, prob, prm, 10, fmt)
    ref, _ = _oracle(lay, prob, prm, 10)
    l1 = G.rel_l1(lay, got, ref)
    assert max(l1) <= TOL_L1, l1
    mags = _magnitudes(lay, prob.U, None, 1.0, 1.0)
    dc = _drift(sums, mags)
    _, sums_plain, _ = _run(torch_cuda, lay, prob, prm, 10, False)
    dp = _drift(sums_plain, mags)
    tol = TOL_DRIFT[fmt]
    assert dc["rho"] <= tol and dc["E_total"] <= tol, (dc, dp)
    assert dc["momentum"] <= tol, (dc, dp)
    assert dc["rho"] < dp["rho"] and dc["E_total"] < dp["E_total"], (dc, dp)


@pytest.mark.parametrize("fmt", ["f32", "i16"])
def test_compensated_rhd_accuracy_and_conservation(torch_cuda, fmt):
    lay, prob, prm = _small_rhd()
    got, sums, st = _run(torch_cuda, lay, prob, prm, 10, fmt)
    assert st[0] == 0, st
    ref_U, ref_R = _oracle(lay, prob, prm, 10)
    l1 = G.rel_l1(lay, got, ref_U + ref_R)
    assert max(l1) <= TOL_L1, l1
    cr = prm["c"] / prm["chat"]
    icc = 1.0 / (prm["c"] * prm["chat"])
    mags = _magnitudes(lay, prob.U, prob.R, cr, icc)
    dc = _drift(sums, mags)
    _, sums_plain, _ = _run(torch_cuda, lay, prob, prm, 10, False)
    dp = _drift(sums_plain, mags)
    tol = TOL_DRIFT[fmt]
    assert dc["rho"] <= tol and dc["E_total"] <= tol, (dc, dp)
    assert dc["momentum"] <= tol, (dc, dp)
    assert dc["E_total"] < dp["E_total"], (dc, dp)

