"""Two-level mesh refinement on the oracle: Berger & Colella (1989) as the
paper applies it (Sec. 2.2 and the level synchronisation of Sec. 2.2.5).

TEST INFRASTRUCTURE ONLY: the plain, slow reference for the library's
refinement path.  Every step of the update on a level is the oracle's own
stage code; this module adds what refinement needs, in numpy, one rule at a
time:

* levels: a coarse patch set covering the periodic domain, and a fine patch
  set (cells a factor 2 smaller) covering part of it, its patches aligned to
  coarse cells;
* one coarse step: dt from both levels (the coarse step is the common step,
  the fine level takes two steps of dt/2; N_sub radiation substeps on each
  level, the same number since dt and the radiation CFL step both halve);
  the coarse level advances first, recording the flux it used at every
  coarse face on the boundary of the fine region; then the fine level takes
  its two steps, its ghost cells outside the fine region filled by
  conservative linear interpolation of the coarse data (readings below),
  recording the fine fluxes at the same boundary;
* synchronisation: each coarse cell next to the fine region gets the
  difference between the fine and the coarse flux integrals through their
  common faces (the flux register), and every coarse cell under the fine
  region is replaced by the mean of its eight fine cells.

Readings (the paper names the methods, not their details):
* interpolation to fine cells: the coarse value plus, per axis, a quarter of
  the monotonized-central slope of the coarse conserved variable (the
  paper's PLM limiter), toward the fine cell; conservative because the eight
  offsets cancel;
* in time, the coarse state is interpolated linearly between the start and
  the end of the coarse step, before the spatial interpolation;
* the flux integral of one RK2-SSP step (hydro step or radiation substep) is
  dt (F(U0) + F(U1)) / 2, the combination the two stages apply; a fine face
  carries a quarter of a coarse face's area.
"""
from __future__ import annotations

import numpy as np

import oracle as O

NHYD, NRAD = 5, 4


def _mc(a, b):
    """Monotonized-central slope of two one-sided differences."""
    s = np.where(a * b > 0.0, 1.0, 0.0)
    m = np.minimum(np.minimum(2.0 * np.abs(a), 2.0 * np.abs(b)), 0.5 * np.abs(a + b))
    return s * np.sign(a + b) * m


class Level:
    def __init__(self, layout, prm):
        self.lay = layout
        self.prm = dict(prm)
        self.p = O.make_params(**self.prm)
        self.g = O.Grid(layout.lo, layout.n, layout.off, layout.dom_n, layout.ng)

    def dense(self, fields):
        """Field arrays -> dense [z, y, x] arrays over the level's domain (zero
        where no patch covers)."""
        out = []
        for f in fields:
            d = np.zeros(tuple(self.lay.dom_n[::-1]))
            for b in range(self.lay.nbox):
                lo, n = self.lay.lo[b], self.lay.n[b]
                d[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]] = \
                    self.lay.interior(f, b)
            out.append(d)
        return out


class TwoLevel:
    """A coarse level covering the periodic domain and one fine level."""

    def __init__(self, coarse_layout, fine_layout, prm):
        cdx = prm.get("dx", 1.0)
        cdx = np.broadcast_to(np.asarray(cdx, dtype=float), (3,))
        self.c = Level(coarse_layout, dict(prm, dx=tuple(cdx)))
        self.f = Level(fine_layout, dict(prm, dx=tuple(cdx / 2.0)))
        cl, fl = coarse_layout, fine_layout
        self.cdom = np.array(cl.dom_n)
        assert np.array_equal(np.array(fl.dom_n), 2 * self.cdom)
        assert np.all(fl.lo % 2 == 0) and np.all(fl.n % 2 == 0)
        # fine coverage on both levels
        fcov = np.zeros(tuple(fl.dom_n[::-1]), dtype=bool)
        for b in range(fl.nbox):
            lo, n = fl.lo[b], fl.n[b]
            fcov[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]] = True
        self.fcov = fcov
        self.ccov = fcov[::2, ::2, ::2].copy()
        self._ghosts()
        self._faces()

    # ------------------------------------------------------------ geometry --
    def _ghosts(self):
        """Per fine patch: the ghost cells no fine patch covers (their indices
        into the patch's full box) and their global fine coordinates."""
        fl, g = self.f.lay, self.f.lay.ng
        fdom = np.array(fl.dom_n)
        self.cf_ghosts = []
        for b in range(fl.nbox):
            n = fl.n[b]
            z, y, x = np.meshgrid(*[np.arange(-g, n[d] + g) for d in (2, 1, 0)], indexing="ij")
            inside = (x >= 0) & (x < n[0]) & (y >= 0) & (y < n[1]) & (z >= 0) & (z < n[2])
            gx = (x + fl.lo[b][0]) % fdom[0]
            gy = (y + fl.lo[b][1]) % fdom[1]
            gz = (z + fl.lo[b][2]) % fdom[2]
            need = ~inside & ~self.fcov[gz, gy, gx]
            self.cf_ghosts.append((need, gx[need], gy[need], gz[need]))

    def _faces(self):
        """The coarse faces on the boundary of the fine region, and the fine
        faces on them.  A coarse face is keyed (d, coarse cell on its high
        side); `out_cell` is the uncovered coarse cell beside it and `side` is
        +1 when that cell lies on the face's low side, -1 on its high side."""
        fl = self.f.lay
        fdom = np.array(fl.dom_n)
        keys = {}
        self.fine_faces = []  # (patch, local cell whose low face it is, d, coarse face id)
        for b in range(fl.nbox):
            lo, n = fl.lo[b], fl.n[b]
            for d in range(3):
                for hi_side in (False, True):
                    # cells of the patch's boundary layer on this side
                    rng = [np.arange(n[a]) for a in range(3)]
                    rng[d] = np.array([n[d] - 1 if hi_side else 0])
                    for cz in rng[2]:
                        for cy in rng[1]:
                            for cx in rng[0]:
                                c = [int(cx), int(cy), int(cz)]
                                nb = list(c)
                                nb[d] += 1 if hi_side else -1
                                gnb = [(nb[a] + lo[a]) % fdom[a] for a in range(3)]
                                if self.fcov[gnb[2], gnb[1], gnb[0]]:
                                    continue
                                # the fine face: low face of its high-side cell
                                hc = nb if hi_side else c
                                ghc = [(hc[a] + lo[a]) % fdom[a] for a in range(3)]
                                chigh = tuple(v // 2 for v in ghc)
                                key = (d, chigh)
                                if key not in keys:
                                    out = list(chigh)
                                    if not hi_side:  # the uncovered cell is on the low side
                                        out[d] = (out[d] - 1) % self.cdom[d]
                                    keys[key] = (len(keys), tuple(out), +1 if not hi_side else -1)
                                self.fine_faces.append((b, tuple(hc), d, keys[key][0]))
        self.nfaces = len(keys)
        self.coarse_faces = [None] * self.nfaces  # (patch, local high-side cell, d)
        self.out_cell = [None] * self.nfaces
        self.side = np.zeros(self.nfaces)
        cl = self.c.lay
        owner = {}
        for q in range(cl.nbox):
            lo, n = cl.lo[q], cl.n[q]
            owner[q] = (lo, n)
        for (d, chigh), (i, out, s) in keys.items():
            for q, (lo, n) in owner.items():
                loc = [chigh[a] - lo[a] for a in range(3)]
                if all(0 <= loc[a] < n[a] for a in range(3)):
                    self.coarse_faces[i] = (q, tuple(loc), d)
                    break
            self.out_cell[i] = out
            self.side[i] = s
        assert all(cf is not None for cf in self.coarse_faces)

    # ------------------------------------------------------ interpolation --
    def fill_cf_ghosts(self, fine_fields, first, cold, cnew, alpha):
        """Fill the fine ghost cells outside the fine region of the given
        fields (state fields first, first+1, ...) from the coarse state at
        (1 - alpha) cold + alpha cnew (dense coarse arrays of all 9 fields)."""
        fl = self.f.lay
        for k, f in enumerate(fine_fields):
            u = (1.0 - alpha) * cold[first + k] + alpha * cnew[first + k]
            slopes = []
            for d in range(3):
                ax = 2 - d
                a = np.roll(u, -1, axis=ax) - u
                bb = u - np.roll(u, 1, axis=ax)
                slopes.append(_mc(a, bb))
            for b in range(fl.nbox):
                need, gx, gy, gz = self.cf_ghosts[b]
                px, py, pz = gx // 2, gy // 2, gz // 2
                v = u[pz, py, px].copy()
                for d, o in enumerate((gx, gy, gz)):
                    sgn = np.where(o % 2 == 0, -0.25, 0.25)
                    v = v + sgn * slopes[d][pz, py, px]
                full = fl.full(f, b)
                full[need] = v

    # ---------------------------------------------------------- registers --
    def _accumulate(self, level, kind, state, rho, weight, reg):
        if level == "c":
            L, faces = self.c, [(cf[0], cf[1], cf[2], i) for i, cf in enumerate(self.coarse_faces)]
            w = weight
        else:
            L, faces = self.f, self.fine_faces
            w = weight * 0.25
        for (b, c, d, i) in faces:
            if kind == "hydro":
                F = O.hydro_face_flux(L.g, L.p, state, b, c, d)
                reg[i, :NHYD] += w * F
            else:
                F = O.rad_face_flux(L.g, L.p, state, rho, b, c, d)
                reg[i, NHYD:] += w * F

    # --------------------------------------------------------- level step --
    def _level_step(self, level, U, R, dt, nsub, dtr, reg, ghosts=None):
        """One step of one level: hydro RK2, then nsub radiation substeps
        with the exchange, fluxes at the register faces accumulated.  ghosts
        (fine level only): callable(fields, first, t_frac) filling the
        fine ghost cells outside the fine region at that fraction of the
        coarse step."""
        L = self.c if level == "c" else self.f
        U1 = [np.zeros_like(a) for a in U]
        if ghosts:
            ghosts(U, 0, 0.0)
        self._accumulate(level, "hydro", U, None, 0.5 * dt, reg)
        O.hydro_stage(L.g, L.p, 1, U, None, U1, dt)
        if ghosts:
            ghosts(U1, 0, 1.0)
        self._accumulate(level, "hydro", U1, None, 0.5 * dt, reg)
        O.hydro_stage(L.g, L.p, 2, U, U1, U, dt)
        if R is None or L.p.hydro_only:
            return
        if ghosts:
            ghosts(U[:1], 0, 1.0)
        R1 = [np.zeros_like(a) for a in R]
        for s in range(nsub):
            if ghosts:
                ghosts(R, NHYD, s / nsub)
            self._accumulate(level, "rad", R, U[0], 0.5 * dtr, reg)
            O.rad_stage(L.g, L.p, 1, R, None, R1, U[0], dtr)
            if ghosts:
                ghosts(R1, NHYD, (s + 1) / nsub)
            self._accumulate(level, "rad", R1, U[0], 0.5 * dtr, reg)
            O.rad_stage(L.g, L.p, 2, R, R1, R, U[0], dtr)
            rc, _ = O.exchange(L.g, L.p, U, R, dtr)
            assert rc == 0, rc

    def timestep(self, Uc, Uf):
        smax = max(O.max_signal_speed(self.c.g, self.c.p, Uc),
                   O.max_signal_speed(self.f.g, self.f.p, Uf))
        return O.timestep_from_speed(self.c.p, smax)

    def step(self, Uc, Rc, Uf, Rf):
        """One coarse step of the two-level hierarchy (in place); returns
        (dt, N_sub)."""
        dt, nsub, dtr = self.timestep(Uc, Uf)
        rad = Rc is not None and not self.c.p.hydro_only
        cold = self.c.dense(Uc + (Rc if rad else [np.zeros_like(Uc[0])] * NRAD))
        reg_c = np.zeros((self.nfaces, NHYD + NRAD))
        reg_f = np.zeros((self.nfaces, NHYD + NRAD))
        self._level_step("c", Uc, Rc if rad else None, dt, nsub, dtr, reg_c)
        cnew = self.c.dense(Uc + (Rc if rad else [np.zeros_like(Uc[0])] * NRAD))
        for k in range(2):
            def ghosts(fields, first, frac, k=k):
                self.fill_cf_ghosts(fields, first, cold, cnew, 0.5 * (k + frac))
            self._level_step("f", Uf, Rf if rad else None, 0.5 * dt, nsub, 0.5 * dtr, reg_f,
                             ghosts)
        self.sync(Uc, Rc if rad else None, Uf, Rf if rad else None, reg_c, reg_f)
        return dt, nsub

    # ---------------------------------------------------------------- sync --
    def sync(self, Uc, Rc, Uf, Rf, reg_c, reg_f):
        cl = self.c.lay
        dxc = np.broadcast_to(np.asarray(self.c.prm["dx"], dtype=float), (3,))
        fields = Uc + (Rc if Rc is not None else [])
        nf = len(fields)
        dense = self.c.dense(fields)
        # reflux: the uncovered coarse cell beside each coarse-fine face
        for i in range(self.nfaces):
            d = self.coarse_faces[i][2]
            x, y, z = self.out_cell[i]
            delta = reg_f[i] - reg_c[i]
            for v in range(nf):
                dense[v][z, y, x] += -self.side[i] * delta[v] / dxc[d]
        # average down: the mean of the eight fine cells
        fdense = self.f.dense(Uf + (Rf if Rf is not None else []))
        for v in range(nf):
            f = fdense[v]
            s = ((f[0::2, 0::2, 0::2] + f[0::2, 0::2, 1::2]) + (f[0::2, 1::2, 0::2] + f[0::2, 1::2, 1::2])) \
                + ((f[1::2, 0::2, 0::2] + f[1::2, 0::2, 1::2]) + (f[1::2, 1::2, 0::2] + f[1::2, 1::2, 1::2]))
            dense[v] = np.where(self.ccov, 0.125 * s, dense[v])
        for v in range(nf):
            for b in range(cl.nbox):
                lo, n = cl.lo[b], cl.n[b]
                cl.interior(fields[v], b)[...] = dense[v][lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1],
                                                          lo[0]:lo[0] + n[0]]

    def totals(self, Uc, Rc, Uf, Rf):
        """Sums over the uncovered coarse cells and the fine cells, times the
        cell volumes: rho, m, E, E_r, F and the RSLA invariants
        E + (c/chat) E_r, m + F/(c chat)."""
        vc = float(np.prod(np.broadcast_to(np.asarray(self.c.prm["dx"], dtype=float), (3,))))
        dc = self.c.dense(Uc + Rc)
        df = self.f.dense(Uf + Rf)
        out = []
        for v in range(NHYD + NRAD):
            out.append(vc * dc[v][~self.ccov].sum() + vc / 8.0 * df[v][self.fcov].sum())
        c, chat = self.c.p.c, self.c.p.chat
        out.append(out[4] + (c / chat) * out[5])
        for a in range(3):
            out.append(out[1 + a] + out[6 + a] / (c * chat))
        return np.array(out)
