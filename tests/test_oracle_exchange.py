"""Pins of the oracle's matter-radiation exchange (Sec. 2.2.3) (no GPU)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
A_R = 7.565767e-15      # radiation constant, erg cm^-3 K^-4 (cgs)
C_LIGHT = 2.99792458e10  # speed of light, cm s^-1


def _closed_form_T4(t, T04, E0, chat_c, a, alpha, kappa, rho, c):
    """Eq. rsla_temperature with E0 = E_g + (c/chat) E_r conserved."""
    Et = E0 / (a + chat_c * alpha / 4.0)
    rate = (4.0 / alpha) * (a + chat_c * alpha / 4.0) * kappa * rho * c
    return (T04 - chat_c * Et) * np.exp(-rate * t) + chat_c * Et


@pytest.mark.parametrize("chat_c", [0.1, 1.0])
def test_exchange_matches_closed_form(chat_c):
    """Sec. 3.2.3: E_r = 1e12, E_g = 1e2, rho = 1e-7, kappa = 1, alpha T^3 heat
    capacity, dt = 1e-8 to t = 1e-2; the temperature agrees with eq.
    rsla_temperature to better than 1 part in 1e5 at every step."""
    gold = json.load(open(os.path.join(GOLD, "paper_values.json")))["exchange"]
    alpha = 4.0 * A_R / gold["epsilon"]
    p = O.make_params(a_r=A_R, c=C_LIGHT, chat=chat_c * C_LIGHT, kappa_P=gold["kappa"],
                      kappa_R=gold["kappa"], eos=1, alpha_eos=alpha, eps_newton=1e-10,
                      max_iter=400)
    nsteps = int(round(gold["t_end"] / gold["dt"]))
    rc, Eg, Er = O.relax_cell(p, gold["rho"], gold["Eg0"], gold["Er0"], gold["dt"], nsteps)
    assert rc == 0
    t = gold["dt"] * np.arange(1, nsteps + 1)
    T04 = 4.0 * gold["Eg0"] / alpha
    E0 = gold["Eg0"] + gold["Er0"] / chat_c
    T4 = _closed_form_T4(t, T04, E0, chat_c, A_R, alpha, gold["kappa"], gold["rho"], C_LIGHT)
    Tnum = (4.0 * Eg / alpha) ** 0.25
    rel = np.abs(Tnum / T4 ** 0.25 - 1.0)
    assert rel.max() < gold["max_rel_error_T"], rel.max()
    # E_0 = E_g + (c/chat) E_r is conserved by every step (Sec. 3.2.3)
    inv = Eg + Er / chat_c
    assert np.abs(np.diff(inv)).max() < 4e-16 * E0  # round-off per step
    assert np.abs(inv / E0 - 1.0).max() < 1e-11     # accumulated over 1e6 steps


def test_rsla_equilibrium_temperature_higher():
    """Sec. 3.2.3: with chat = 0.1 c the RSLA equilibrium temperature is about
    20 per cent above the physically correct one (closed form: ratio
    (T_eq,RSLA / T_eq)^4 = (chat/c) E0_RSLA (a + alpha/4) / (E0 (a + (chat/c) alpha/4)))."""
    gold = json.load(open(os.path.join(GOLD, "paper_values.json")))["exchange"]
    alpha = 4.0 * A_R
    Teq = {}
    for chat_c in (0.1, 1.0):
        p = O.make_params(a_r=A_R, c=C_LIGHT, chat=chat_c * C_LIGHT, kappa_P=1.0, kappa_R=1.0,
                          eos=1, alpha_eos=alpha)
        rc, Eg, Er = O.relax_cell(p, gold["rho"], gold["Eg0"], gold["Er0"], gold["dt"], 1000000)
        assert rc == 0
        Teq[chat_c] = (4.0 * Eg[-1] / alpha) ** 0.25
    ratio = Teq[0.1] / Teq[1.0]
    assert abs(ratio - gold["Teq_ratio_approx"]) < 0.06, ratio
    E0r = gold["Eg0"] + 10.0 * gold["Er0"]
    E0c = gold["Eg0"] + gold["Er0"]
    exact = (0.1 * E0r / (A_R + 0.1 * alpha / 4) / (E0c / (A_R + alpha / 4))) ** 0.25
    assert abs(ratio / exact - 1.0) < 1e-6


def _bisect_Eg(p, rho, Eg0, Er0, dt):
    """Root of the single-variable form of F_G = F_R = 0: eliminating E_r with
    F_R = 0 gives R = k (a T^4 - E_r0)/(1 + k), k = dt rho kappa chat, and then
    g(E_g) = E_g - E_g0 + (c/chat) R(E_g) = 0, increasing in E_g."""
    k = dt * rho * p.kappa_P * p.chat
    cr = p.c / p.chat

    def g(Eg):
        T = Eg / (rho * p.c_v)
        return Eg - Eg0 + cr * k * (p.a_r * T ** 4 - Er0) / (1 + k)

    lo, hi = 0.0, Eg0 + cr * Er0
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            hi = mid
        else:
            lo = mid
    Eg = 0.5 * (lo + hi)
    T = Eg / (rho * p.c_v)
    Er = (Er0 + k * p.a_r * T ** 4) / (1 + k)
    return Eg, Er


def test_newton_matches_bisection():
    """The Newton iteration of eqs. delta_er and delta_eg converges to the
    unique root of the backward-Euler system (checked by bisection on the
    equivalent scalar equation) across non-stiff and stiff cells."""
    rng = np.random.Generator(np.random.Philox(17))
    p = O.make_params(gamma=5 / 3, a_r=1.0, c=100.0, chat=10.0, kappa_P=1.0)
    for _ in range(400):
        rho = math.exp(rng.uniform(-4, 4))
        Eg0 = rho * p.c_v * math.exp(rng.uniform(-1, 1))
        Er0 = math.exp(rng.uniform(-3, 3))
        dt = math.exp(rng.uniform(-9, -1))
        Eg, Er, it = O.exchange_energy(p, rho, Eg0, Er0, dt)
        assert it > 0
        Egb, Erb = _bisect_Eg(p, rho, Eg0, Er0, dt)
        Etot = Eg0 + (p.c / p.chat) * Er0
        assert abs(Eg - Egb) < 1e-12 * Etot, (rho, Eg0, Er0, dt)
        assert abs(Er - Erb) * (p.c / p.chat) < 1e-12 * Etot


def test_newton_reports_nonconvergence():
    """Sec. 2.2.3: exceeding the iteration limit is an error (a status, not an
    exit): a stiff cell with max_iter = 1 reports -1 / ENOCONV."""
    p = O.make_params(a_r=1.0, c=100.0, chat=10.0, kappa_P=1.0, max_iter=1)
    assert O.exchange_energy(p, 1.0, 1.5, 16.0, 0.1)[2] == -1
    lay = I.single_box(2, 2, 2)
    U = I.zeros(lay, 5)
    R = I.zeros(lay, 4)
    lay.interior(U[0], 0)[...] = 1.0
    lay.interior(U[4], 0)[...] = 1.5
    lay.interior(R[0], 0)[...] = 16.0
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    rc, info = O.exchange(g, p, U, R, 0.1)
    assert rc == O.ENOCONV and info[0] & (1 << O.ENOCONV) and info[1] >= 0


def test_exchange_invariants_per_cell():
    """Per cell, the exchange conserves E + (c/chat) E_r (the energy terms
    of eqs. hydro_energy and rad_energy plus the work term move energy
    between them in that ratio) and m + F/(c chat) (the equal and opposite
    momentum update), to round-off; F relaxes monotonically towards 0."""
    lay = I.single_box(6, 5, 4)
    rng = np.random.Generator(np.random.Philox(23))
    U = I.zeros(lay, 5)
    R = I.zeros(lay, 4)
    shp = lay.interior(U[0], 0).shape
    rho = np.exp(rng.uniform(-2, 2, shp))
    v = 0.5 * rng.standard_normal((3,) + shp)
    Eg = rho * 1.5 * rng.uniform(0.5, 2.0, shp)
    lay.interior(U[0], 0)[...] = rho
    for d in range(3):
        lay.interior(U[1 + d], 0)[...] = rho * v[d]
    lay.interior(U[4], 0)[...] = Eg + 0.5 * rho * (v ** 2).sum(0)
    Er = rng.uniform(0.1, 10.0, shp)
    lay.interior(R[0], 0)[...] = Er
    f = 0.5 * rng.standard_normal((3,) + shp)
    for d in range(3):
        lay.interior(R[1 + d], 0)[...] = 100.0 * Er * f[d]
    p = O.make_params(gamma=5 / 3, a_r=1.0, c=100.0, chat=10.0, kappa_P=1.0, kappa_R=2.0,
                      kappa_mode=1)
    inv_E = lambda: lay.interior(U[4], 0) + 10.0 * lay.interior(R[0], 0)
    inv_m = lambda d: lay.interior(U[1 + d], 0) + lay.interior(R[1 + d], 0) / 1000.0
    e0 = inv_E().copy()
    m0 = [inv_m(d).copy() for d in range(3)]
    F0 = [lay.interior(R[1 + d], 0).copy() for d in range(3)]
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    rc, info = O.exchange(g, p, U, R, 0.01)
    assert rc == 0 and info[2] <= 10
    assert np.abs(inv_E() / e0 - 1.0).max() < 1e-14
    scale = np.abs(np.array(F0)).max() / 1000.0
    for d in range(3):
        assert np.abs(inv_m(d) - m0[d]).max() < 1e-14 * scale
        Fn = lay.interior(R[1 + d], 0)
        assert np.all(np.abs(Fn) <= np.abs(F0[d])) and np.all(Fn * F0[d] >= 0)
