"""Small seeded or closed-form initial states for the tests (1-D problems run on
an N x 1 x 1 periodic grid along any axis, 3-D random states), shared by the
oracle pins and the GPU parity tests.  Nothing here computes a step of the
update."""
from __future__ import annotations

import numpy as np

from paper_2110_01792_gb300 import inputs as I


def line_layout(N, axis=0, ng=4):
    n = [1, 1, 1]
    n[axis] = N
    return I.make_layout([[0, 0, 0]], [n], tuple(n), ng)


def set_line(lay, arr, values, axis):
    """Write a length-N profile along ``axis`` into the interior of patch 0."""
    v = lay.interior(arr, 0)
    shape = [1, 1, 1]
    shape[2 - axis] = len(values)
    v[...] = np.asarray(values, dtype=arr.dtype).reshape(shape)


def get_line(lay, arr, axis):
    return lay.interior(arr, 0).reshape(-1).copy()


def hydro_line(N, rho, u, p, gamma, axis=0, ng=4, vt=(0.0, 0.0)):
    """1-D hydro state with normal velocity u along ``axis``; vt are the two
    transverse velocities (axis+1, axis+2 mod 3)."""
    lay = line_layout(N, axis, ng)
    U = I.zeros(lay, 5)
    rho = np.broadcast_to(np.asarray(rho, dtype=float), (N,))
    u = np.broadcast_to(np.asarray(u, dtype=float), (N,))
    p = np.broadcast_to(np.asarray(p, dtype=float), (N,))
    vel = [None, None, None]
    vel[axis] = u
    vel[(axis + 1) % 3] = np.full(N, vt[0])
    vel[(axis + 2) % 3] = np.full(N, vt[1])
    set_line(lay, U[0], rho, axis)
    for d in range(3):
        set_line(lay, U[1 + d], rho * vel[d], axis)
    ke = 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    set_line(lay, U[4], p / (gamma - 1.0) + ke, axis)
    return lay, U


def centres(N, L=1.0):
    return (np.arange(N) + 0.5) * (L / N)


def random_hydro_3d(n, seed=7, ng=4, lay=None, vamp=0.3):
    """Random smooth-ish 3-D periodic hydro state (positive rho and P)."""
    if lay is None:
        lay = I.single_box(*n, ng=ng) if isinstance(n, (tuple, list)) else I.single_box(n, ng=ng)
    rng = np.random.Generator(np.random.Philox(seed))
    gamma = 5.0 / 3.0
    U = I.zeros(lay, 5)
    for b in range(lay.nbox):
        shp = lay.interior(U[0], b).shape
        rho = 1.0 + 0.3 * rng.random(shp)
        v = vamp * rng.standard_normal((3,) + shp)
        P = 1.0 + 0.3 * rng.random(shp)
        lay.interior(U[0], b)[...] = rho
        for d in range(3):
            lay.interior(U[1 + d], b)[...] = rho * v[d]
        lay.interior(U[4], b)[...] = P / (gamma - 1.0) + 0.5 * rho * (v ** 2).sum(0)
    return lay, U, gamma


def random_rad_3d(lay, seed=11, fmax=0.6):
    """Random radiation state with |f| <= fmax."""
    rng = np.random.Generator(np.random.Philox(seed))
    R = I.zeros(lay, 4)
    c = 100.0
    for b in range(lay.nbox):
        shp = lay.interior(R[0], b).shape
        Er = 0.5 + rng.random(shp)
        f = rng.standard_normal((3,) + shp)
        f *= fmax * rng.random(shp) / np.maximum(np.sqrt((f ** 2).sum(0)), 1e-12)
        lay.interior(R[0], b)[...] = Er
        for d in range(3):
            lay.interior(R[1 + d], b)[...] = c * Er * f[d]
    return R


# cgs constants (CODATA), used by the problems the paper states in cgs units
A_RAD = 7.5657e-15      # radiation constant, erg cm^-3 K^-4
C_LIGHT = 2.99792458e10  # cm s^-1
K_B = 1.380649e-16      # erg K^-1
M_H = 1.6735575e-24     # hydrogen atom mass, g


def radiation_pressure_tube(spec, N=None, ng=4):
    """Sec. 3.3.1: the steady state of radiation and gas pressure in the
    equilibrium-diffusion limit.  T(x), rho(x) solve
        d rho/dx = -(mu/(k T)) (k rho/mu + (4/3) a_r T^3) dT/dx,
        d2T/dx2  = -(3/T) (dT/dx)^2 + (1/rho) (d rho/dx)(dT/dx)
    from T0, rho0, drho0/dx at x = 0 (``spec``: the golden entry), integrated
    with scipy over the interior and the ghost cells; E_r = a_r T^4, the flux is
    the diffusion flux F = -(c/(3 kappa rho)) dE_r/dx, the gas is at rest.  The
    ghost cells hold the same solution (the Dirichlet boundary states).
    Returns (layout, U, R, params, T_exact at the interior cells)."""
    from scipy.integrate import solve_ivp
    N = int(spec["N"]) if N is None else N
    L = float(spec["L"])
    dx = L / N
    mu = spec["mu_over_mH"] * M_H
    gamma = spec["gamma"]
    kappa = spec["kappa"]
    T0, rho0, drho0 = spec["T0"], spec["rho0"], spec["drho0_dx"]

    def rhs(x, y):
        rho, T, Tp = y
        drho = -(mu / (K_B * T)) * (K_B * rho / mu + 4.0 / 3.0 * A_RAD * T ** 3) * Tp
        return [drho, Tp, -3.0 / T * Tp ** 2 + drho / rho * Tp]

    Tp0 = -drho0 / ((mu / (K_B * T0)) * (K_B * rho0 / mu + 4.0 / 3.0 * A_RAD * T0 ** 3))
    xc = (np.arange(-ng, N + ng) + 0.5) * dx
    right = solve_ivp(rhs, (0.0, xc[-1]), [rho0, T0, Tp0], rtol=1e-12, atol=1e-30,
                      dense_output=True)
    left = solve_ivp(rhs, (0.0, xc[0]), [rho0, T0, Tp0], rtol=1e-12, atol=1e-30,
                     dense_output=True)
    rho, T, Tp = np.array([left.sol(x) if x < 0 else right.sol(x) for x in xc]).T
    cv = K_B / ((gamma - 1.0) * mu)
    cs0 = np.sqrt(gamma * K_B * T0 / mu)
    lay = line_layout(N, 0, ng)
    U = I.zeros(lay, 5)
    R = I.zeros(lay, 4)
    for arr, vals in ((U[0], rho), (U[4], rho * cv * T), (R[0], A_RAD * T ** 4),
                      (R[1], -(C_LIGHT / (3 * kappa * rho)) * 4 * A_RAD * T ** 3 * Tp)):
        lay.full(arr, 0)[...] = vals[None, None, :]
    params = dict(gamma=gamma, cfl=spec["cfl"], a_r=A_RAD, c=C_LIGHT,
                  chat=spec["chat_over_cs0"] * cs0, c_v=cv, kappa_P=kappa, kappa_R=kappa,
                  dx=dx, bc_lo=(3, 0, 0), bc_hi=(3, 0, 0), nsub_max=10, tau_correction=1)
    return lay, U, R, params, T[ng:N + ng], L / cs0


# --------------------------------------------- dense whole-domain states ---
VEC_AXIS = {1: 0, 2: 1, 3: 2, 6: 0, 7: 1, 8: 2}  # state field id -> vector axis


def scatter(lay, dense):
    """Dense [z, y, x] arrays of the whole domain -> field arrays of a layout."""
    out = I.zeros(lay, len(dense))
    for f, d in zip(out, dense):
        for b in range(lay.nbox):
            lo, n = lay.lo[b], lay.n[b]
            lay.interior(f, b)[...] = d[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]]
    return out


def gather(lay, fields):
    out = []
    for f in fields:
        d = np.zeros(tuple(lay.dom_n[::-1]))
        for b in range(lay.nbox):
            lo, n = lay.lo[b], lay.n[b]
            d[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]] = lay.interior(f, b)
        out.append(d)
    return out


def two_patches(n, ng=4):
    """The domain n split into two patches along x (non-equal widths)."""
    a = n[0] // 2 + 1
    return I.make_layout([[0, 0, 0], [a, 0, 0]], [[a, n[1], n[2]], [n[0] - a, n[1], n[2]]],
                         tuple(n), ng)


def random_state(n, seed, rad=True):
    """Dense random RHD state (rho, m, E, E_r, F) on a domain n = (nx, ny, nz)."""
    rng = np.random.Generator(np.random.Philox(seed))
    shp = (n[2], n[1], n[0])
    rho = np.exp(0.4 * rng.standard_normal(shp))
    v = 0.5 * rng.standard_normal((3,) + shp)
    P = np.exp(0.3 * rng.standard_normal(shp))
    gamma = 5.0 / 3.0
    U = [rho, rho * v[0], rho * v[1], rho * v[2], P / (gamma - 1) + 0.5 * rho * (v ** 2).sum(0)]
    if not rad:
        return U
    Er = np.exp(0.3 * rng.standard_normal(shp))
    f = rng.standard_normal((3,) + shp)
    f *= 0.7 * rng.random(shp) / np.sqrt((f ** 2).sum(0))
    c = 20.0
    return U + [Er, c * Er * f[0], c * Er * f[1], c * Er * f[2]]


def mirror_double(dense, axes):
    """Append the mirror image along each axis in ``axes`` (0 = x); vector
    components along that axis change sign in the image."""
    out = list(dense)
    for ax in axes:
        npax = 2 - ax
        out = [np.concatenate([d, (-1.0 if VEC_AXIS.get(fid) == ax else 1.0) * np.flip(d, npax)],
                              axis=npax) for fid, d in enumerate(out)]
    return out


def blob_in_ambient(n, pad, margin, seed):
    """A random blob inside a uniform ambient state: ``margin`` ambient cells
    between the blob and each non-periodic wall, ``pad`` more ambient cells
    beyond the walls (the padded periodic twin)."""
    ambient = [1.0, 0.3, -0.2, 0.1, 2.0, 1.0, 2.0, -1.0, 0.5]
    shp = (n[2] + 2 * pad[2], n[1] + 2 * pad[1], n[0] + 2 * pad[0])
    dense = [np.full(shp, v) for v in ambient]
    m = [margin if p else 0 for p in pad]
    blob = random_state(tuple(n[d] - 2 * m[d] for d in range(3)), seed)
    sl = tuple(slice(pad[d] + m[d], pad[d] + n[d] - m[d]) for d in (2, 1, 0))
    for d, b in zip(dense, blob):
        d[sl] = b
    return dense


def random_state_smooth(lay, seed, amp=0.3, c=20.0):
    """Smooth periodic RHD state on a layout: a few random low-order Fourier
    modes (Philox-seeded) per field, evaluated at cell centres of the domain
    [0, 1)^3 scaled by dom_n; positive rho, P, E_r and |f| <= 0.6."""
    rng = np.random.Generator(np.random.Philox(seed))
    dom = np.array(lay.dom_n, dtype=float)
    modes = []
    for _ in range(9):
        k = rng.integers(-2, 3, size=(3, 3))
        ph = rng.uniform(0, 2 * np.pi, size=3)
        a = rng.uniform(0.3, 1.0, size=3)
        modes.append((k, ph, a))

    def field(v, X, Y, Z):
        k, ph, a = modes[v]
        s = np.zeros_like(X)
        for m in range(3):
            s += a[m] * np.sin(2 * np.pi * (k[m, 0] * X + k[m, 1] * Y + k[m, 2] * Z) + ph[m])
        return s / 3.0

    gamma = 5.0 / 3.0
    U = I.zeros(lay, 5)
    R = I.zeros(lay, 4)
    for b in range(lay.nbox):
        lo, n = lay.lo[b], lay.n[b]
        Z, Y, X = np.meshgrid(*[(lo[d] + np.arange(n[d]) + 0.5) / dom[d] for d in (2, 1, 0)],
                              indexing="ij")
        rho = np.exp(amp * field(0, X, Y, Z))
        v = [amp * field(1 + d, X, Y, Z) for d in range(3)]
        P_ = np.exp(amp * field(4, X, Y, Z))
        Er = np.exp(amp * field(5, X, Y, Z))
        f = [0.2 * field(6 + d, X, Y, Z) for d in range(3)]
        lay.interior(U[0], b)[...] = rho
        for d in range(3):
            lay.interior(U[1 + d], b)[...] = rho * v[d]
        lay.interior(U[4], b)[...] = P_ / (gamma - 1) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
        lay.interior(R[0], b)[...] = Er
        for d in range(3):
            lay.interior(R[1 + d], b)[...] = c * Er * f[d]
    return U, R


def refine_state(coarse, fine, fields):
    """Fine fields from coarse ones by injection: every fine cell takes its
    coarse parent's value (a newly refined level before its first step)."""
    dense = gather(coarse, fields)
    out = [np.zeros(fine.field_len) for _ in fields]
    for f, d in zip(out, dense):
        for b in range(fine.nbox):
            lo, n = fine.lo[b], fine.n[b]
            idx = [((lo[a] + np.arange(n[a])) // 2) % coarse.dom_n[a] for a in range(3)]
            fine.interior(f, b)[...] = d[np.ix_(idx[2], idx[1], idx[0])]
    return out[:5], out[5:]
