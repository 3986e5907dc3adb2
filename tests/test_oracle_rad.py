"""Pins of the oracle's radiation stage and closure (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from tests import problems as P


def _grid(lay):
    return O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)


# ------------------------------------------------------------ closure -----

def test_levermore_closure_limits():
    """Eq. M1_closure: chi(0) = 1/3 gives the isotropic tensor I/3; chi(1) = 1
    gives the streaming tensor n n; the trace is always 1; chi is the
    eigenvalue along n and is monotone in |f|."""
    T = O.eddington_tensor([0.0, 0.0, 0.0])
    np.testing.assert_allclose(T, np.eye(3) / 3.0, rtol=0, atol=1e-16)
    n = np.array([1.0, 2.0, -2.0]) / 3.0
    T = O.eddington_tensor(n)
    np.testing.assert_allclose(T, np.outer(n, n), atol=1e-15)
    prev = 1.0 / 3.0
    rng = np.random.Generator(np.random.Philox(1))
    for fm in np.linspace(0.01, 1.0, 60):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        T = O.eddington_tensor(fm * d)
        assert abs(np.trace(T) - 1.0) < 1e-14
        np.testing.assert_allclose(T, T.T, atol=0)
        chi = d @ T @ d
        chi_ref = (3 + 4 * fm ** 2) / (5 + 2 * math.sqrt(4 - 3 * fm ** 2))
        assert abs(chi - chi_ref) < 1e-14
        assert chi >= prev - 1e-15
        prev = chi
        # transverse eigenvalue (1 - chi)/2
        e = np.cross(d, [0.3, -0.1, 0.9])
        e /= np.linalg.norm(e)
        assert abs(e @ T @ e - 0.5 * (1 - chi)) < 1e-14


def test_closure_rescales_superluminal_flux():
    """|f| > 1 is rescaled to |f| = 1 for the closure only (Sec. 2.2.2)."""
    d = np.array([0.6, 0.0, 0.8])
    np.testing.assert_allclose(O.eddington_tensor(1.7 * d), O.eddington_tensor(d), atol=1e-15)


# -------------------------------------------------- transport pulses ------

def _rad_run(lay, p, R, rho, t_end, exchange_U=None):
    g = _grid(lay)
    R1 = [np.zeros_like(a) for a in R]
    t = 0.0
    dxm = min(p.dx)
    dtr = p.cfl * dxm / p.chat
    n = 0
    while t < t_end * (1 - 1e-14):
        dt = min(dtr, t_end - t)
        O.rad_stage(g, p, 1, R, None, R1, rho, dt)
        O.rad_stage(g, p, 2, R, R1, R, rho, dt)
        if exchange_U is not None:
            rc, _ = O.exchange(g, p, exchange_U, R, dt)
            assert rc == 0
        t += dt
        n += 1
    return n


def _pulse_1d(N, axis, E0, A, sig, fx, c, x0=0.5):
    lay = P.line_layout(N, axis)
    R = I.zeros(lay, 4)
    x = P.centres(N)
    E = E0 + A * np.exp(-0.5 * ((x - x0) / sig) ** 2)
    P.set_line(lay, R[0], E, axis)
    P.set_line(lay, R[1 + axis], c * E * fx, axis)
    rho = np.zeros(lay.field_len)
    lay.interior(rho, 0)[...] = 1.0
    return lay, R, rho, x


@pytest.mark.parametrize("axis", [0, 2])
def test_free_streaming_pulse_translates(axis):
    """kappa = 0 and |f| = 1: eqs. rad_energy and rad_flux reduce to linear
    advection of E_r at speed chat (the Levermore tensor is n n), so the exact
    solution is a translation.  The pulse centroid moves at chat, F stays
    c E_r, and the L1 error falls with resolution.  (At |f| = 1 exactly,
    rounding noise puts some face states at |f| = 1 + 1 ulp, which the
    first-order fallback of Sec. 2.2.2 treats as a violation, so the error
    converges at less than the design order here.)"""
    errs = []
    for N in (64, 128, 256):
        c, chat = 10.0, 1.0
        lay, R, rho, x = _pulse_1d(N, axis, 1.0, 1.0, 0.06, 1.0, c)
        dx = [1.0, 1.0, 1.0]
        dx[axis] = 1.0 / N
        p = O.make_params(c=c, chat=chat, kappa_P=0.0, kappa_R=0.0, cfl=0.3, dx=dx,
                          tau_correction=1)
        t = 0.25
        E_init = P.get_line(lay, R[0], axis)
        _rad_run(lay, p, R, rho, t)
        E = P.get_line(lay, R[0], axis)
        ex = 1.0 + np.exp(-0.5 * (((x - 0.5 - chat * t + 0.5) % 1.0 - 0.5) / 0.06) ** 2)
        errs.append(np.abs(E - ex).mean())
        F = P.get_line(lay, R[1 + axis], axis)
        assert np.abs(F - c * E).max() < 1e-9 * c
        cen0 = ((E_init - 1.0) * x).sum() / (E_init - 1.0).sum()
        cen1 = ((E - 1.0) * x).sum() / (E - 1.0).sum()
        assert abs((cen1 - cen0) - chat * t) < 1e-2 * chat * t, (N, cen1 - cen0)
        assert abs(E.sum() - E_init.sum()) < 1e-12 * E.sum()
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[0] / errs[2] > 3.0, errs
    assert errs[-1] < 1.5e-2, errs


@pytest.mark.parametrize("N", [64, 128, 256])
def test_diffusion_limit_gaussian(N):
    """Optically thick, kappa_P = 0: eq. rad_flux with the backward-Euler flux
    source of Sec. 2.2.3 drives F to -(c/(3 rho kappa_R)) dE/dx, so E_r obeys
    dE/dt = D d2E/dx2 with D = chat/(3 rho kappa_R) and a Gaussian pulse
    spreads with variance sigma0^2 + 2 D t.  For the split scheme (one RK2-SSP
    transport substep, then the flux source) the modified equation gives
    D_eff = D (1 + k/2), k = chat rho kappa_R dt_rad = rho kappa_R CFL dx,
    which tends to D as the mean free path is resolved.  The measured
    variance growth must match D_eff within 2 %: a wrong c, chat or rho kappa
    factor in the flux or the source moves it by far more.  The gas is heavy
    (rho = 1e6 at the same rho kappa_R) so that the radiation force and its
    kinetic-energy work term stay negligible without a hydro update."""
    c, chat, rk, cfl = 10.0, 1.0, 400.0, 0.3
    rho0 = 1e6
    sig0 = 0.04
    lay, R, rho, x = _pulse_1d(N, 0, 1.0, 1.0, sig0, 0.0, c)
    rho *= rho0
    U = I.zeros(lay, 5)
    lay.interior(U[0], 0)[...] = rho0
    lay.interior(U[4], 0)[...] = 1.0
    p = O.make_params(c=c, chat=chat, kappa_P=0.0, kappa_R=rk / rho0, cfl=cfl, dx=1.0 / N,
                      tau_correction=1, gamma=5 / 3)
    D = chat / (3.0 * rk)
    k = rk * cfl / N
    Deff = D * (1.0 + 0.5 * k)
    t = 1.5 * sig0 ** 2 / (2 * D)
    E0 = P.get_line(lay, R[0], 0).sum()
    _rad_run(lay, p, R, rho, t, exchange_U=U)
    E = P.get_line(lay, R[0], 0)
    assert abs(E.sum() - E0) < 1e-6 * E0  # only the tiny kinetic-energy work term
    w = E - 1.0
    var = (w * (x - 0.5) ** 2).sum() / w.sum()
    assert abs((var - sig0 ** 2) / (2 * t) / Deff - 1.0) < 0.02, ((var - sig0 ** 2) / (2 * t), Deff)
    s2 = sig0 ** 2 + 2 * Deff * t
    ex = 1.0 + (sig0 / math.sqrt(s2)) * np.exp(-0.5 * (x - 0.5) ** 2 / s2)
    assert np.abs(E - ex).max() < 0.02 * (ex.max() - 1.0)


def test_radiation_conservation_periodic():
    """With no source terms, the flux form conserves sum E_r and sum F to
    round-off on a periodic patch set."""
    lay = I.make_layout([[0, 0, 0], [8, 0, 0]], [[8, 6, 5], [4, 6, 5]], (12, 6, 5), 4)
    R = P.random_rad_3d(lay, seed=3)
    rho = np.zeros(lay.field_len)
    for b in range(lay.nbox):
        lay.interior(rho, b)[...] = 1.0 + np.arange(lay.interior(rho, b).size).reshape(
            lay.interior(rho, b).shape) % 3
    U = I.zeros(lay, 5)
    U[0][:] = rho
    p = O.make_params(c=100.0, chat=10.0, kappa_P=1.0, kappa_R=1.0, cfl=0.3, dx=1.0 / 12)
    g = _grid(lay)
    s0 = O.conserved_sums(g, p, U, R)
    R1 = [np.zeros_like(a) for a in R]
    for _ in range(4):
        O.rad_stage(g, p, 1, R, None, R1, rho, 1e-3)
        O.rad_stage(g, p, 2, R, R1, R, rho, 1e-3)
    s1 = O.conserved_sums(g, p, U, R)
    assert abs(s1[5] - s0[5]) <= 1e-14 * abs(s0[5])
    for v in (6, 7, 8):
        assert abs(s1[v] - s0[v]) <= 1e-14 * 100.0 * abs(s0[5])


def test_radiation_uniform_state_unchanged():
    """A uniform radiation state with any flux |f| < 1 is a fixed point."""
    lay = I.single_box(6, 5, 4)
    R = I.zeros(lay, 4)
    vals = [2.0, 100.0 * 2.0 * 0.3, -100.0 * 2.0 * 0.2, 100.0 * 2.0 * 0.1]
    for a, v in zip(R, vals):
        lay.interior(a, 0)[...] = v
    R0 = [a.copy() for a in R]
    rho = np.ones(lay.field_len)
    p = O.make_params(c=100.0, chat=10.0, cfl=0.3, dx=1.0 / 6)
    g = _grid(lay)
    R1 = [np.zeros_like(a) for a in R]
    O.rad_stage(g, p, 1, R, None, R1, rho, 1e-3)
    O.rad_stage(g, p, 2, R, R1, R, rho, 1e-3)
    for a, b in zip(R, R0):
        assert np.array_equal(lay.interior(a, 0), lay.interior(b, 0))


@pytest.mark.parametrize("tau_cell", [0.0, 4.0])
def test_single_step_at_an_energy_jump_closed_form(tau_cell):
    """One forward stage of the radiation update at a jump of E_r (1 | 2)
    with a uniform reduced flux f = (0.3, 0, 0), by hand: PLM keeps the face
    states at the cell averages there (the MC slopes vanish beside a step),
    so the HLL flux at the jump face is
      energy: (chat/2) f (E_L + E_R) - (S eps / 2)(E_R - E_L),
      F_x:    (c chat/2) chi (E_L + E_R) - (S eps c f / 2)(E_R - E_L),
    with S = chat sqrt(T_xx) = chat sqrt(chi) of the cell averages (Levermore
    chi(0.3), the same on both sides) and eps = min(1, 1/tau), tau = dx (rho
    kappa_R) (Sec. 2.2.2; the optical-depth factor as read), and the faces
    inside the two plateaus carry the upwind-free flux of the uniform state.
    A dropped 1/2, chat/c, square root or eps changes the cells beside the
    jump at O(dt/dx)."""
    N = 16
    lay = I.single_box(N, 4, 4)
    c, chat, f0, dt = 100.0, 10.0, 0.3, 1e-3
    dx = 1.0 / N
    R = I.zeros(lay, 4)
    E = np.where(np.arange(N) < N // 2, 1.0, 2.0)
    lay.interior(R[0], 0)[...] = E[None, None, :]
    lay.interior(R[1], 0)[...] = c * f0 * E[None, None, :]
    kap = tau_cell / dx
    rho = np.ones(lay.field_len)
    p = O.make_params(c=c, chat=chat, kappa_P=kap, kappa_R=kap, dx=dx, recon=1,
                      tau_correction=1)
    g = _grid(lay)
    R1 = [np.zeros_like(a) for a in R]
    O.rad_stage(g, p, 1, R, None, R1, rho, dt)
    chi = (3.0 + 4.0 * f0 ** 2) / (5.0 + 2.0 * math.sqrt(4.0 - 3.0 * f0 ** 2))
    S = chat * math.sqrt(chi)
    eps = 1.0 if tau_cell <= 1.0 else 1.0 / tau_cell
    EL, ER = 1.0, 2.0
    FE = 0.5 * chat * f0 * (EL + ER) - 0.5 * S * eps * (ER - EL)
    FF = 0.5 * c * chat * chi * (EL + ER) - 0.5 * S * eps * c * f0 * (ER - EL)
    k = dt / dx
    want = {  # cell: (E, F_x) after the stage
        N // 2 - 1: (EL - k * (FE - chat * f0 * EL), c * f0 * EL - k * (FF - c * chat * chi * EL)),
        N // 2: (ER - k * (chat * f0 * ER - FE), c * f0 * ER - k * (c * chat * chi * ER - FF)),
        N // 4: (EL, c * f0 * EL),
    }
    Eo, Fo = lay.interior(R1[0], 0), lay.interior(R1[1], 0)
    for i, (we, wf) in want.items():
        assert np.allclose(Eo[:, :, i], we, rtol=1e-13, atol=0), (i, Eo[0, 0, i], we)
        assert np.allclose(Fo[:, :, i], wf, rtol=1e-13, atol=0), (i, Fo[0, 0, i], wf)
        assert np.all(lay.interior(R1[2], 0)[:, :, i] == 0.0)
