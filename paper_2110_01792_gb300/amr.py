"""Two-level mesh refinement step on the GPU (Berger & Colella 1989, as Sec.
2.2 and its level synchronisation apply it), composed from the library's
entry points: every operation runs in the CUDA kernels of libqk; this module
only orders the calls and keeps the coarse state at the start of the step
(for the fine ghost cells' interpolation in time).

One coarse step: the common dt from both levels (qk_signal_speed on each,
qk_set_timestep on the coarse one); the coarse level's hydro RK2 step and
N_sub radiation substeps with the exchange, the flux at the coarse-fine
faces recorded before each stage; then two fine steps of dt/2 (the same
N_sub), each stage preceded by the fine ghost fill and the interpolation of
the fine ghost cells outside the fine region at that stage's time, with the
fine fluxes recorded; finally the level synchronisation (reflux, average
down)."""
from __future__ import annotations

from . import qk


class AmrStepper:
    def __init__(self, coarse_layout, fine_layout, params: dict, precision: int = qk.FP64):
        import numpy as np
        dx = np.broadcast_to(np.asarray(params.get("dx", 1.0), dtype=float), (3,))
        self.cctx = qk.Context(coarse_layout, dict(params, dx=tuple(dx)), precision)
        self.fctx = qk.Context(fine_layout, dict(params, dx=tuple(dx / 2.0)), precision, level=True)
        self.amr = qk.Amr(self.cctx, self.fctx)
        self._scratch = {}

    def close(self):
        self.amr.close()
        self.fctx.close()
        self.cctx.close()

    def _tmp(self, key, like):
        import torch
        if key not in self._scratch:
            self._scratch[key] = [torch.empty_like(a) for a in like]
        return self._scratch[key]

    def step(self, Uc, Rc, Uf, Rf):
        """One coarse step in place; returns (dt, N_sub)."""
        cc, fc, amr = self.cctx, self.fctx, self.amr
        smax = max(cc.signal_speed(Uc), fc.signal_speed(Uf))
        dt, nsub, dtr, _ = cc.set_timestep(smax)
        rad = Rc is not None and not cc.params.hydro_only
        cfields = Uc + (Rc if rad else [])
        cc.fill_ghosts(cfields, 0)
        cold = self._tmp("cold", cfields)
        for a, b in zip(cold, cfields):
            a.copy_(b)
        cold9 = cold + [None] * (9 - len(cold))
        self._level(cc, 0, Uc, Rc if rad else None, dt, nsub, dtr, None)
        cc.fill_ghosts(cfields, 0)
        cnew9 = cfields + [None] * (9 - len(cfields))
        for k in range(2):
            def ghosts(fields, first, frac, k=k):
                amr.interp(cold9, cnew9, 0.5 * (k + frac), fields, first)
            self._level(fc, 1, Uf, Rf if rad else None, 0.5 * dt, nsub, 0.5 * dtr, ghosts)
        amr.sync(Uc, Rc if rad else None, Uf, Rf if rad else None)
        return dt, nsub

    def _level(self, ctx, lev, U, R, dt, nsub, dtr, ghosts):
        amr = self.amr
        U1 = self._tmp(("U1", lev), U)
        ctx.fill_ghosts(U, 0)
        if ghosts:
            ghosts(U, 0, 0.0)
        ctx.hydro_stage(1, U, None, U1, dt)
        amr.register(lev, 0, U, None, 0.5 * dt)
        ctx.fill_ghosts(U1, 0)
        if ghosts:
            ghosts(U1, 0, 1.0)
        ctx.hydro_stage(2, U, U1, U, dt)
        amr.register(lev, 0, U1, None, 0.5 * dt)
        if R is None:
            return
        R1 = self._tmp(("R1", lev), R)
        ctx.fill_ghosts(U[:1], 0)
        if ghosts:
            ghosts(U[:1], 0, 1.0)
        for s in range(nsub):
            ctx.fill_ghosts(R, 5)
            if ghosts:
                ghosts(R, 5, s / nsub)
            ctx.rad_stage(1, R, None, R1, U[0], dtr)
            amr.register(lev, 1, R, U[0], 0.5 * dtr)
            ctx.fill_ghosts(R1, 5)
            if ghosts:
                ghosts(R1, 5, (s + 1) / nsub)
            ctx.rad_stage(2, R, R1, R, U[0], dtr)
            amr.register(lev, 1, R1, U[0], 0.5 * dtr)
            ctx.exchange(U, R, dtr)
