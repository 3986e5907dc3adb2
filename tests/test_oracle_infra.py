"""Pins of the oracle's ghost fill, patch handling, sums and whole step."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from tests import problems as P


def _grid(lay):
    return O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)


def test_ghost_fill_single_box_is_periodic_wrap():
    """A single periodic box: ghost cells equal numpy's wrap padding."""
    lay = I.single_box(7, 5, 6, ng=4)
    rng = np.random.Generator(np.random.Philox(2))
    f = np.zeros(lay.field_len)
    inner = rng.standard_normal((6, 5, 7))
    lay.interior(f, 0)[...] = inner
    O.fill_ghosts(_grid(lay), f)
    assert np.array_equal(lay.full(f, 0), np.pad(inner, 4, mode="wrap"))


def test_ghost_fill_thin_axes_multiple_wraps():
    """Extents smaller than the ghost width wrap more than once."""
    lay = I.single_box(9, 1, 2, ng=4)
    f = np.zeros(lay.field_len)
    inner = np.arange(18, dtype=float).reshape(2, 1, 9)
    lay.interior(f, 0)[...] = inner
    O.fill_ghosts(_grid(lay), f)
    assert np.array_equal(lay.full(f, 0), np.pad(inner, 4, mode="wrap"))


def test_ghost_fill_patch_tiling_matches_global_array():
    """A random guillotine tiling: every patch's ghost layer equals the
    corresponding periodic slice of the assembled global array."""
    lay = I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=3, edges=(8, 16, 24))
    assert lay.nbox > 4
    rng = np.random.Generator(np.random.Philox(4))
    glob = rng.standard_normal(lay.dom_n[::-1])
    f = np.zeros(lay.field_len)
    for b in range(lay.nbox):
        lo, n = lay.lo[b], lay.n[b]
        lay.interior(f, b)[...] = glob[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]]
    O.fill_ghosts(_grid(lay), f)
    padded = np.pad(glob, 3, mode="wrap")
    for b in range(lay.nbox):
        lo, n = lay.lo[b], lay.n[b]
        ref = padded[lo[2]:lo[2] + n[2] + 6, lo[1]:lo[1] + n[1] + 6, lo[0]:lo[0] + n[0] + 6]
        assert np.array_equal(lay.full(f, b), ref)


def test_patch_tiling_covers_domain_once():
    lay = I.patch_tiling()
    cover = np.zeros(lay.dom_n[::-1], dtype=np.int16)
    for b in range(lay.nbox):
        lo, n = lay.lo[b], lay.n[b]
        assert all(int(v) in (16, 24, 32, 48, 64) for v in n)
        cover[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]] += 1
    assert cover.min() == 1 and cover.max() == 1
    assert 1200 < lay.nbox < 1900
    assert np.all(lay.off % I.PAD == 0)


def test_conserved_sums_match_fsum():
    """Compensated sums agree with math.fsum (exactly rounded) to 1 ulp."""
    lay = I.make_layout([[0, 0, 0], [4, 0, 0]], [[4, 3, 2], [5, 3, 2]], (9, 3, 2), 2)
    rng = np.random.Generator(np.random.Philox(8))
    U = I.zeros(lay, 5)
    R = I.zeros(lay, 4)
    for a in U + R:
        for b in range(lay.nbox):
            lay.interior(a, b)[...] = rng.standard_normal(lay.interior(a, b).shape) * 1e3
    p = O.make_params(c=100.0, chat=10.0, dx=(0.5, 0.25, 2.0))
    s = O.conserved_sums(_grid(lay), p, U, R)
    vals = lambda a: np.concatenate([lay.interior(a, b).ravel() for b in range(lay.nbox)])
    fields = [vals(a) for a in U + R]
    ref = [math.fsum(f) for f in fields]
    ref.append(math.fsum(fields[4] + 10.0 * fields[5]))
    for d in range(3):
        ref.append(math.fsum(fields[1 + d] + fields[6 + d] / 1000.0))
    vol = 0.5 * 0.25 * 2.0
    for got, r in zip(s, ref):
        assert abs(got - r * vol) <= 2e-16 * max(abs(r * vol), 1.0)


def test_rhd_step_conserves_rsla_invariants():
    """Whole RHD step on a periodic patch set: sum rho is conserved, and so
    are sum(E + (c/chat) E_r) and sum(m + F/(c chat)), the quantities the
    transport conserves in flux form and the exchange conserves per cell
    (eqs. hydro_continuity..rad_flux, Sec. 2.2.3)."""
    lay = I.make_layout([[0, 0, 0], [8, 0, 0], [0, 8, 0]],
                        [[8, 8, 8], [4, 12, 8], [8, 4, 8]], (12, 12, 8), 4)
    prob = I.rhd_lognormal(layout=lay, seed=3)
    U, R = prob.U, prob.R
    prm = dict(prob.params)
    prm["dx"] = 1.0 / 12
    p = O.make_params(**prm)
    g = _grid(lay)
    s0 = O.conserved_sums(g, p, U, R)
    rc, ts, info = O.step(g, p, U, R)
    assert rc == 0 and ts[1] >= 1 and info[2] < 50
    rc, ts, info = O.step(g, p, U, R)
    assert rc == 0
    s1 = O.conserved_sums(g, p, U, R)
    assert abs(s1[0] - s0[0]) <= 1e-14 * abs(s0[0])
    assert abs(s1[9] - s0[9]) <= 1e-13 * abs(s0[9])
    mscale = abs(s0[9]) / 100.0
    for d in range(3):
        assert abs(s1[10 + d] - s0[10 + d]) <= 1e-13 * mscale


def test_planted_sign_error_is_caught():
    """A plausible mistake must fail a pin: flipping the sign of the HLLC
    momentum flux breaks the stationary-contact and consistency pins
    (demonstrated here on the oracle's own formulas, on the CPU)."""
    wl = [1.0, 0.3, 0.0, 0.0, 1.0]
    F = O.hllc(wl, wl, 0, 1.4)
    bad = F.copy()
    bad[1] = -bad[1]
    E = 1.0 / 0.4 + 0.5 * 0.09
    good = [0.3, 0.09 + 1.0, 0.0, 0.0, 0.3 * (E + 1.0)]
    np.testing.assert_allclose(F, good, rtol=1e-14)
    assert not np.allclose(bad, good)


@pytest.mark.parametrize("flat,bc", [(0, "periodic"), (1, "walls")])
def test_threaded_oracle_is_bit_identical(flat, bc):
    """The oracle's host-thread cell loops (z-planes over OpenMP threads)
    change no arithmetic: three RHD steps of a ragged patch set on 1 and on
    several threads give the same bits in every field, the same timestep and
    the same exchange record (status, first failing cell, iterations)."""
    lay = I.patch_tiling(dom_n=(24, 16, 16), seed=7, ng=4, edges=(8, 16))
    prob = I.rhd_lognormal(layout=lay, seed=9, kappa_mode=1, sigma=1.5)
    prm = dict(prob.params, dx=1.0 / 24, flattening=flat)
    if bc == "walls":
        prm.update(bc_lo=(O.BC_REFLECT, 0, 0), bc_hi=(O.BC_OUTFLOW, 0, 0))
    g = _grid(lay)
    p = O.make_params(**prm)
    results = []
    try:
        for nt in (1, 4):
            O.set_threads(nt)
            U = [a.copy() for a in prob.U]
            R = [a.copy() for a in prob.R]
            recs = [O.step(g, p, U, R) for _ in range(3)]
            results.append((U + R, recs))
    finally:
        O.set_threads(1)
    (f1, r1), (f4, r4) = results
    assert r1 == r4
    for a, b in zip(f1, f4):
        np.testing.assert_array_equal(a, b)
