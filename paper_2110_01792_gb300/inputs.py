"""Seeded synthetic inputs for the per-cell uniform-patch RHD update.

This module holds no step of the update itself: it only lays out patches in
memory, draws seeded random initial states and writes them as conserved
variables.  Both the CUDA path and the CPU oracle are fed from here.

Layout (shared by the library and the oracle): every field is one contiguous
array over all patches; patch ``b`` starts at element ``off[b]`` (a multiple of
64 elements) and holds ``(n_x+2g)(n_y+2g)(n_z+2g)`` cells, x fastest.

Workloads (all periodic, cells on [0,1)^3 scaled by 1/n):
  * ``hydro_waves`` -- density 1 + 0.1 sum_k a_k sin(2 pi n_k.x + phi_k) over 8
    integer wavevectors with 0 < |n_k| <= 4, a_k ~ U(0,1)/8, phi_k ~ U(0,2pi),
    uniform P = 1, velocities N(0, 0.1^2) per cell; gamma = 5/3, CFL 0.3.
  * ``rhd_lognormal`` -- ln rho = sigma g - sigma^2/2 with g a unit-variance
    Gaussian random field of power spectrum |k|^-4 (P(0) = 0); v = 0, uniform
    gas temperature T = 1, E_r = a_r T_r^4 with T_r ~ U(0.5, 2), F = 0;
    kappa_P = kappa_R = 1 (or kappa0 rho), a_r = 1, c = 100,
    chat = 10 max c_s at t = 0.  These stand in for the paper's Sedov and
    radiation-driven-shell performance problems (Sec. 4), which are not
    distributed as data.
  * ``patch_tiling`` -- a guillotine random tiling of a periodic domain into
    boxes with edges drawn from {16, 24, 32, 48, 64}.
Random numbers come from numpy's counter-based Philox generator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PAD = 64  # patch offsets are multiples of this many elements


@dataclass
class Layout:
    lo: np.ndarray  # (nbox, 3) int32, patch lower corner in the domain
    n: np.ndarray  # (nbox, 3) int32, interior extents
    off: np.ndarray  # (nbox,) int64, element offset of each patch
    ng: int
    dom_n: tuple
    field_len: int

    @property
    def nbox(self) -> int:
        return len(self.off)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n.astype(np.int64), axis=1).sum())

    def patch_shape(self, b):
        nx, ny, nz = (int(v) + 2 * self.ng for v in self.n[b])
        return nz, ny, nx

    def interior(self, arr: np.ndarray, b: int) -> np.ndarray:
        """View of patch b's interior cells, indexed [k, j, i]."""
        nz, ny, nx = self.patch_shape(b)
        g = self.ng
        v = arr[self.off[b]:self.off[b] + nx * ny * nz].reshape(nz, ny, nx)
        n = self.n[b]
        return v[g:g + n[2], g:g + n[1], g:g + n[0]]

    def full(self, arr: np.ndarray, b: int) -> np.ndarray:
        nz, ny, nx = self.patch_shape(b)
        return arr[self.off[b]:self.off[b] + nx * ny * nz].reshape(nz, ny, nx)


def make_layout(lo, n, dom_n, ng: int) -> Layout:
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1, 3)
    n = np.ascontiguousarray(n, dtype=np.int32).reshape(-1, 3)
    offs = np.zeros(len(n), dtype=np.int64)
    pos = 0
    for b in range(len(n)):
        offs[b] = pos
        vol = int(np.prod(n[b].astype(np.int64) + 2 * ng))
        pos += (vol + PAD - 1) // PAD * PAD
    return Layout(lo, n, offs, int(ng), tuple(int(v) for v in dom_n), int(pos))


def single_box(nx, ny=None, nz=None, ng=4) -> Layout:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return make_layout([[0, 0, 0]], [[nx, ny, nz]], (nx, ny, nz), ng)


def split_line(rng, length, edges=(16, 24, 32, 48, 64)):
    """Split a periodic line into segments from ``edges``; a draw is redone
    while it would leave a remainder that is neither 0 nor >= min(edges)."""
    out = []
    rem = length
    lo = min(edges)
    while rem > 0:
        ok = [e for e in edges if e <= rem and (rem - e == 0 or rem - e >= lo)]
        if not ok:
            raise ValueError(f"cannot split length {length} into {edges}")
        e = int(rng.choice(ok))
        out.append(e)
        rem -= e
    return out


def patch_tiling(dom_n=(512, 384, 384), seed=2110, ng=4,
                 edges=(16, 24, 32, 48, 64)) -> Layout:
    """Guillotine random tiling: x slabs, y columns per slab, z bricks per column."""
    rng = np.random.Generator(np.random.Philox(seed))
    los, ns = [], []
    x0 = 0
    for wx in split_line(rng, dom_n[0], edges):
        y0 = 0
        for wy in split_line(rng, dom_n[1], edges):
            z0 = 0
            for wz in split_line(rng, dom_n[2], edges):
                los.append([x0, y0, z0])
                ns.append([wx, wy, wz])
                z0 += wz
            y0 += wy
        x0 += wx
    return make_layout(los, ns, dom_n, ng)


def zeros(layout: Layout, nf: int, dtype=np.float64):
    return [np.zeros(layout.field_len, dtype=dtype) for _ in range(nf)]


def _rng(seed, *keys):
    ss = np.random.SeedSequence([int(seed)] + [int(k) for k in keys])
    return np.random.Generator(np.random.Philox(ss))


def _centres(n):
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    return np.meshgrid(z, y, x, indexing="ij")  # Z, Y, X with shape (nz, ny, nx)


def gaussian_random_field(rng, shape_zyx, slope=-4.0):
    """Unit-variance periodic Gaussian random field with P(k) ~ |k|^slope, P(0)=0."""
    noise = rng.standard_normal(shape_zyx)
    fk = np.fft.rfftn(noise)
    kz = np.fft.fftfreq(shape_zyx[0]) * shape_zyx[0]
    ky = np.fft.fftfreq(shape_zyx[1]) * shape_zyx[1]
    kx = np.fft.rfftfreq(shape_zyx[2]) * shape_zyx[2]
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = np.zeros_like(K2)
    nz = K2 > 0
    amp[nz] = K2[nz] ** (slope / 4.0)  # sqrt(P) = |k|^(slope/2)
    g = np.fft.irfftn(fk * amp, s=shape_zyx, axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


@dataclass
class Problem:
    """A workload: layout, physical parameters, initial conserved state."""
    name: str
    layout: Layout
    params: dict
    U: list
    R: list | None = None
    steps: int = 10
    meta: dict = field(default_factory=dict)


def hydro_waves(n=32, seed=2110, ng=4, layout: Layout | None = None, steps=10) -> Problem:
    """Hydro-only smooth-density / noisy-velocity periodic state (gamma = 5/3)."""
    lay = layout or single_box(n, ng=ng)
    gamma = 5.0 / 3.0
    U = zeros(lay, 5)
    dom = np.array(lay.dom_n)
    for b in range(lay.nbox):
        rng_modes = _rng(seed, 0)
        rng_v = _rng(seed, 1, b)
        nvec = []
        while len(nvec) < 8:
            v = rng_modes.integers(-4, 5, size=3)
            m2 = int((v * v).sum())
            if 0 < m2 <= 16:
                nvec.append(v)
        a = rng_modes.uniform(0.0, 1.0, size=8) / 8.0
        phi = rng_modes.uniform(0.0, 2 * math.pi, size=8)
        nb = lay.n[b]
        z = (lay.lo[b][2] + np.arange(nb[2]) + 0.5) / dom[2]
        y = (lay.lo[b][1] + np.arange(nb[1]) + 0.5) / dom[1]
        x = (lay.lo[b][0] + np.arange(nb[0]) + 0.5) / dom[0]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        rho = np.ones_like(X)
        for kk in range(8):
            rho += 0.1 * a[kk] * np.sin(2 * math.pi * (nvec[kk][0] * X + nvec[kk][1] * Y +
                                                       nvec[kk][2] * Z) + phi[kk])
        P = np.ones_like(X)
        v = rng_v.normal(0.0, 0.1, size=(3,) + X.shape)
        lay.interior(U[0], b)[...] = rho
        for d in range(3):
            lay.interior(U[1 + d], b)[...] = rho * v[d]
        lay.interior(U[4], b)[...] = P / (gamma - 1.0) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    params = dict(gamma=gamma, cfl=0.3, dx=1.0 / dom[0], hydro_only=1)
    return Problem("hydro_waves", lay, params, U, None, steps)


def rhd_lognormal(n=128, seed=2110, ng=4, sigma=1.0, kappa_mode=0, kappa0=1.0,
                  layout: Layout | None = None, steps=20) -> Problem:
    """RHD lognormal-density state with out-of-equilibrium radiation."""
    lay = layout or single_box(n, ng=ng)
    gamma = 5.0 / 3.0
    c_v = 1.0 / (gamma - 1.0)
    a_r, c = 1.0, 100.0
    T_gas = 1.0
    U = zeros(lay, 5)
    R = zeros(lay, 4)
    for b in range(lay.nbox):
        rng = _rng(seed, 2, b)
        nb = lay.n[b]
        shape = (int(nb[2]), int(nb[1]), int(nb[0]))
        g = gaussian_random_field(rng, shape)
        rho = np.exp(sigma * g - 0.5 * sigma * sigma)
        Tr = rng.uniform(0.5, 2.0, size=shape)
        lay.interior(U[0], b)[...] = rho
        lay.interior(U[4], b)[...] = rho * c_v * T_gas
        lay.interior(R[0], b)[...] = a_r * Tr ** 4
    cs0 = math.sqrt(gamma * (gamma - 1.0) * c_v * T_gas)
    params = dict(gamma=gamma, cfl=0.3, dx=1.0 / lay.dom_n[0], a_r=a_r, c=c, chat=10.0 * cs0,
                  c_v=c_v, kappa_P=kappa0, kappa_R=kappa0, kappa_mode=kappa_mode,
                  eps_newton=1e-10, max_iter=400, nsub_max=10, tau_correction=1,
                  hydro_only=0)
    return Problem("rhd_lognormal", lay, params, U, R, steps,
                   dict(sigma=sigma, seed=seed))


def config(name: str, **kw) -> Problem:
    """The named workloads of the benchmark and the parity tests."""
    if name == "hydro32":
        return hydro_waves(32, steps=10, **kw)
    if name == "rhd128":
        return rhd_lognormal(128, steps=20, **kw)
    if name == "hydro256":
        return hydro_waves(256, steps=10, **kw)
    if name == "rhd256":
        return rhd_lognormal(256, steps=20, **kw)
    if name == "rhd512":
        return rhd_lognormal(512, sigma=1.5, kappa_mode=1, steps=10, **kw)
    if name == "patches":
        lay = patch_tiling()
        return rhd_lognormal(layout=lay, steps=10, **kw)
    raise KeyError(name)
