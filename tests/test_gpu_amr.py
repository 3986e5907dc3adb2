"""GPU parity of two-level mesh refinement: the library's refinement
operations (interpolation of the fine ghost cells, flux registers, reflux,
average down) driven by paper_2110_01792_gb300.amr against the oracle's
two-level hierarchy (oracle/amr.py) on the same seeded inputs: FP64 to 1e-10
per cell after 3 coarse steps on both levels, conservation to round-off on
the GPU, FP32-mixed within 1e-5 relative L1."""
import numpy as np
import pytest

from oracle.amr import TwoLevel
from tests import gpu_util as G
from tests import problems as P
from tests.test_oracle_amr import PRM, hierarchy

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


def _initial(seed=3):
    coarse, fine = hierarchy()
    Uc, Rc = P.random_state_smooth(coarse, seed)
    Uf, Rf = P.refine_state(coarse, fine, Uc + Rc)
    return coarse, fine, Uc, Rc, Uf, Rf


def _run_gpu(prm, nsteps, prec=0, rad=True, seed=3):
    torch = pytest.importorskip("torch")
    from paper_2110_01792_gb300.amr import AmrStepper
    coarse, fine, Uc, Rc, Uf, Rf = _initial(seed)
    dt = torch.float64 if prec == 0 else torch.float32
    st = AmrStepper(coarse, fine, prm, prec)
    dUc, dUf = G.dev(Uc, dt), G.dev(Uf, dt)
    dRc, dRf = (G.dev(Rc, dt), G.dev(Rf, dt)) if rad else (None, None)
    hist = [st.step(dUc, dRc, dUf, dRf) for _ in range(nsteps)]
    torch.cuda.synchronize()
    info = st.amr.info()
    status = (st.cctx.status(), st.fctx.status())
    st.close()
    out = (G.host(dUc), G.host(dRc) if rad else None, G.host(dUf), G.host(dRf) if rad else None)
    return out, hist, info, status


def _run_oracle(prm, nsteps, rad=True, seed=3):
    coarse, fine, Uc, Rc, Uf, Rf = _initial(seed)
    h = TwoLevel(coarse, fine, prm)
    hist = [h.step(Uc, Rc if rad else None, Uf, Rf if rad else None) for _ in range(nsteps)]
    return (Uc, Rc if rad else None, Uf, Rf if rad else None), hist, h


def _err(lay, got, ref):
    return G.max_rel_err(lay, got, ref)


@pytest.mark.parametrize("variant", ["rhd", "rhd_plm_flat", "hydro"])
def test_amr_steps_match_oracle(torch_cuda, variant):
    """3 coarse steps of the L-shaped two-level hierarchy (coarse RHD step
    with 5 radiation substeps, two fine steps, reflux, average down): every
    cell of both levels agrees with the oracle to 1e-10; dt and N_sub agree;
    the list sizes match the oracle's geometry; no Newton failure."""
    prm = dict(PRM)
    rad = variant != "hydro"
    if variant == "rhd_plm_flat":
        prm.update(recon=1, flattening=1)
    if not rad:
        prm.update(hydro_only=1)
    (gUc, gRc, gUf, gRf), hg, info, status = _run_gpu(prm, 3, rad=rad)
    (oUc, oRc, oUf, oRf), ho, h = _run_oracle(prm, 3, rad=rad)
    assert status[0][0] == 0 and status[1][0] == 0, status
    for (dg, ng_), (do, no) in zip(hg, ho):
        assert abs(dg - do) <= 1e-13 * do and int(ng_) == int(no)
    ncf = sum(int(c[0].sum()) for c in h.cf_ghosts)
    assert info == (ncf, h.nfaces, int(h.ccov.sum())), (info, ncf, h.nfaces)
    coarse, fine = hierarchy()
    ec = _err(coarse, gUc + (gRc or []), oUc + (oRc or []))
    ef = _err(fine, gUf + (gRf or []), oUf + (oRf or []))
    assert max(ec) <= 1e-10 and max(ef) <= 1e-10, (ec, ef)


def test_amr_conserves_on_gpu(torch_cuda):
    """The GPU hierarchy conserves rho, E + (c/chat) E_r and m + F/(c chat)
    to round-off over 3 refined RHD steps (sums over the uncovered coarse
    cells and the fine cells)."""
    coarse, fine, Uc, Rc, Uf, Rf = _initial()
    h = TwoLevel(coarse, fine, PRM)
    t0 = h.totals(Uc, Rc, Uf, Rf)
    (gUc, gRc, gUf, gRf), _, _, _ = _run_gpu(dict(PRM), 3)
    t1 = h.totals(gUc, gRc, gUf, gRf)
    assert abs(t1[0] - t0[0]) <= 1e-14 * abs(t0[0])
    assert abs(t1[9] - t0[9]) <= 1e-13 * abs(t0[9])
    for a in range(3):
        assert abs(t1[10 + a] - t0[10 + a]) <= 1e-13 * abs(t0[9]) / 20.0


def test_amr_mixed_precision(torch_cuda):
    """FP32-mixed hierarchy: relative L1 error of rho, E and E_r on both
    levels against the FP64 oracle <= 1e-5 after 3 coarse steps."""
    (gUc, gRc, gUf, gRf), _, _, status = _run_gpu(dict(PRM), 3, prec=1)
    coarse, fine, Uc, Rc, Uf, Rf = _initial()
    Uc = [a.astype(np.float32).astype(np.float64) for a in Uc]
    Rc = [a.astype(np.float32).astype(np.float64) for a in Rc]
    Uf = [a.astype(np.float32).astype(np.float64) for a in Uf]
    Rf = [a.astype(np.float32).astype(np.float64) for a in Rf]
    h = TwoLevel(coarse, fine, PRM)
    for _ in range(3):
        h.step(Uc, Rc, Uf, Rf)
    assert status[0][0] == 0 and status[1][0] == 0
    lc = G.rel_l1(coarse, [gUc[0], gUc[4], gRc[0]], [Uc[0], Uc[4], Rc[0]])
    lf = G.rel_l1(fine, [gUf[0], gUf[4], gRf[0]], [Uf[0], Uf[4], Rf[0]])
    assert max(lc + lf) <= 1e-5, (lc, lf)
