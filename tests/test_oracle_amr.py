"""Pins of the oracle's two-level mesh refinement (no GPU): conservation to
round-off through the flux register and averaging down (Berger & Colella
1989, the level synchronisation of Sec. 2.2.5), conservative and
linear-exact interpolation, a uniform state kept exactly, and a refined wave
more accurate than the coarse one."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.amr import TwoLevel
from paper_2110_01792_gb300 import inputs as I
from tests import problems as P


def hierarchy(ng=4):
    """Coarse 16 x 12 x 8 in two patches; fine region: two fine patches
    covering coarse cells [4, 12) x [2, 10) x [2, 6) and [12, 14) x [2, 6) x
    [2, 6) (an L-shaped region: fine-fine neighbours and concave corners)."""
    coarse = P.two_patches((16, 12, 8), ng)
    fine = I.make_layout([[8, 4, 4], [24, 4, 4]], [[16, 16, 8], [4, 8, 8]], (32, 24, 16), ng)
    return coarse, fine


def _state(lay, seed, amp=0.3):
    U, R = P.random_state_smooth(lay, seed, amp)
    return U, R


PRM = dict(gamma=5.0 / 3.0, cfl=0.3, c=20.0, chat=4.0, kappa_P=2.0, kappa_R=3.0, a_r=1.0,
           c_v=1.5, dx=1.0 / 16)


def _setup(seed=3, **kw):
    coarse, fine = hierarchy()
    h = TwoLevel(coarse, fine, dict(PRM, **kw))
    Uc, Rc = _state(coarse, seed)
    # the fine level starts from the conservative interpolation of the coarse
    # state (every fine cell from its coarse parent, like a newly refined grid)
    Uf, Rf = P.refine_state(coarse, fine, Uc + Rc)
    return h, Uc, Rc, Uf, Rf


def test_refined_steps_conserve_to_roundoff():
    """Three coarse steps (each: coarse hydro + 5 radiation substeps + exchange,
    two fine steps, reflux, average down) on the periodic two-level
    hierarchy: the sums of rho, E + (c/chat) E_r and m + F/(c chat) over the
    uncovered coarse cells and the fine cells change by round-off only.  The
    same steps without the flux register lose conservation by orders of
    magnitude more, so the pin sees a missing or mis-signed correction."""
    h, Uc, Rc, Uf, Rf = _setup()
    t0 = h.totals(Uc, Rc, Uf, Rf)
    nsubs = [h.step(Uc, Rc, Uf, Rf)[1] for _ in range(3)]
    assert max(nsubs) >= 2
    t1 = h.totals(Uc, Rc, Uf, Rf)
    assert abs(t1[0] - t0[0]) <= 1e-14 * abs(t0[0])
    assert abs(t1[9] - t0[9]) <= 1e-13 * abs(t0[9])
    scale = abs(t0[9]) / 20.0
    for a in range(3):
        assert abs(t1[10 + a] - t0[10 + a]) <= 1e-13 * scale
    # without the register: drop the reflux term
    h2, Uc2, Rc2, Uf2, Rf2 = _setup()
    sync = h2.sync
    h2.sync = lambda Uc_, Rc_, Uf_, Rf_, rc, rf: sync(Uc_, Rc_, Uf_, Rf_, rc, rc)
    for _ in range(3):
        h2.step(Uc2, Rc2, Uf2, Rf2)
    t2 = h2.totals(Uc2, Rc2, Uf2, Rf2)
    assert abs(t2[0] - t0[0]) > 1e3 * abs(t1[0] - t0[0]) + 1e-12 * abs(t0[0])


def test_interpolation_is_conservative_and_linear_exact():
    """The fine ghost cells outside the fine region: every 2x2x2 block of
    ghost cells that fills one coarse cell averages to that coarse cell's
    value (to round-off), and a linear coarse field (away from the periodic
    seam) is reproduced exactly at the fine cell centres."""
    coarse, fine = hierarchy()
    h = TwoLevel(coarse, fine, PRM)
    rng = np.random.Generator(np.random.Philox(8))
    dense = [rng.standard_normal((8, 12, 16)) for _ in range(9)]
    fields = [np.zeros(fine.field_len) for _ in range(9)]
    h.fill_cf_ghosts(fields, 0, dense, dense, 0.0)
    g = fine.ng
    for b in range(fine.nbox):
        need, gx, gy, gz = h.cf_ghosts[b]
        full = [fine.full(f, b) for f in fields]
        # blocks: ghost cells with even global coordinates and their 7 partners
        sel = (gx % 2 == 0) & (gy % 2 == 0) & (gz % 2 == 0)
        idx = np.argwhere(need)[sel]
        for (z, y, x) in idx[:200]:
            if z + 1 >= full[0].shape[0] or y + 1 >= full[0].shape[1] or x + 1 >= full[0].shape[2]:
                continue
            if not need[z:z + 2, y:y + 2, x:x + 2].all():
                continue
            px = ((x - g + fine.lo[b][0]) % 32) // 2
            py = ((y - g + fine.lo[b][1]) % 24) // 2
            pz = ((z - g + fine.lo[b][2]) % 16) // 2
            for v in range(9):
                m = full[v][z:z + 2, y:y + 2, x:x + 2].mean()
                assert abs(m - dense[v][pz, py, px]) <= 1e-14 * (1 + abs(dense[v][pz, py, px]))
    # linear field: exact in the interior of the coarse domain
    zc, yc, xc = np.meshgrid(np.arange(8), np.arange(12), np.arange(16), indexing="ij")
    lin = [0.3 + 0.02 * xc - 0.05 * yc + 0.07 * zc] * 9
    fields = [np.zeros(fine.field_len) for _ in range(9)]
    h.fill_cf_ghosts(fields, 0, lin, lin, 0.0)
    for b in range(fine.nbox):
        need, gx, gy, gz = h.cf_ghosts[b]
        ok = (gx >= 2) & (gx < 30) & (gy >= 2) & (gy < 22) & (gz >= 2) & (gz < 14)
        exact = 0.3 + 0.02 * (gx + 0.5) / 2 - 0.02 * 0.5 - 0.05 * ((gy + 0.5) / 2 - 0.5) \
            + 0.07 * ((gz + 0.5) / 2 - 0.5)
        got = fine.full(fields[0], b)[need]
        assert np.abs(got[ok] - exact[ok]).max() < 1e-14


def test_uniform_state_stays_uniform():
    """A uniform moving gas with uniform radiation stays uniform on both
    levels after refined steps: every interpolation and flux sees uniform
    data; the flux register's sums of equal fine and coarse flux integrals
    cancel to round-off (sums of 16 equal terms round), hence 1e-14."""
    coarse, fine = hierarchy()
    h = TwoLevel(coarse, fine, dict(PRM, kappa_P=0.0, kappa_R=0.0))
    vals = [1.2, 0.3, -0.2, 0.1, 3.0, 1.5, 2.0, -1.0, 0.5]
    Uc = [np.full(coarse.field_len, v) for v in vals[:5]]
    Rc = [np.full(coarse.field_len, v) for v in vals[5:]]
    Uf = [np.full(fine.field_len, v) for v in vals[:5]]
    Rf = [np.full(fine.field_len, v) for v in vals[5:]]
    for _ in range(2):
        h.step(Uc, Rc, Uf, Rf)
    for a, v in zip(Uc + Rc, vals):
        for b in range(coarse.nbox):
            assert np.abs(coarse.interior(a, b) - v).max() <= 1e-14 * 3.0
    for a, v in zip(Uf + Rf, vals):
        for b in range(fine.nbox):
            assert np.abs(fine.interior(a, b) - v).max() <= 1e-14 * 3.0


def _wave_error(levels):
    """Sound wave along x (Sec. 3.1.1 eigenvector, amplitude 1e-4) on a
    32 x 4 x 4 coarse grid, optionally refined on x in [8, 24); L1 error of
    rho after one period against the exact translation, per cell volume."""
    g = 5.0 / 3.0
    N = 32
    coarse = I.make_layout([[0, 0, 0]], [[N, 4, 4]], (N, 4, 4), 4)
    x = P.centres(N)
    A = 1e-4
    cs = 1.0
    P0 = 1.0 / g

    def state(lay, xs):
        U = I.zeros(lay, 5)
        for b in range(lay.nbox):
            lo, n = lay.lo[b], lay.n[b]
            xx = xs[lo[0]:lo[0] + n[0]]
            rho = 1.0 + A * np.sin(2 * math.pi * xx)
            u = A * cs * np.sin(2 * math.pi * xx)
            p = P0 + A * g * P0 * np.sin(2 * math.pi * xx)
            lay.interior(U[0], b)[...] = rho[None, None, :]
            lay.interior(U[1], b)[...] = (rho * u)[None, None, :]
            lay.interior(U[4], b)[...] = (p / (g - 1) + 0.5 * rho * u * u)[None, None, :]
        return U

    prm = dict(gamma=g, cfl=0.3, dx=1.0 / N, hydro_only=1)
    Uc = state(coarse, x)
    R0 = [np.ones(coarse.field_len)] + [np.zeros(coarse.field_len)] * 3
    if levels == 1:
        grid = O.Grid(coarse.lo, coarse.n, coarse.off, coarse.dom_n, coarse.ng)
        p = O.make_params(**prm)
        t = 0.0
        while t < 1.0 - 1e-12:
            dt = min(O.timestep(grid, p, Uc)[0], 1.0 - t)
            U1 = [np.zeros_like(a) for a in Uc]
            O.hydro_stage(grid, p, 1, Uc, None, U1, dt)
            O.hydro_stage(grid, p, 2, Uc, U1, Uc, dt)
            t += dt
        got = P.gather(coarse, [Uc[0]])[0][0, 0, :]
        return np.abs(got - (1.0 + A * np.sin(2 * math.pi * (x - t)))).mean() / A
    fine = I.make_layout([[16, 0, 0]], [[32, 8, 8]], (2 * N, 8, 8), 4)
    h = TwoLevel(coarse, fine, prm)
    Uf, _ = P.refine_state(coarse, fine, Uc + R0)
    Rf = None
    t = 0.0
    while t < 1.0 - 1e-12:
        dt, _ = h.step(Uc, None, Uf, None)
        t += dt
    # the hierarchy steps to t >= 1: compare at the time it reached
    rc = h.c.dense(Uc)[0][0, 0, :]
    rf = h.f.dense(Uf)[0][0, 0, :]
    err = 0.0
    xf = P.centres(2 * N)
    for i in range(N):
        if h.ccov[0, 0, i]:
            continue
        err += abs(rc[i] - (1.0 + A * np.sin(2 * math.pi * (x[i] - t))))
    for i in range(16, 48):
        err += 0.5 * abs(rf[i] - (1.0 + A * np.sin(2 * math.pi * (xf[i] - t))))
    return err / N / A


@pytest.mark.slow
def test_refined_wave_beats_the_coarse_grid():
    """Refining the middle half of a sound wave's path lowers its L1 error
    after one period below the coarse-only error: the interface neither
    reflects nor distorts the wave at this level."""
    e1 = _wave_error(1)
    e2 = _wave_error(2)
    assert e2 < 0.85 * e1, (e1, e2)
