"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas, written from the mathematics of Toro (2009), ch. 4: the pressure
function f_K(p) (shock branch from the Rankine-Hugoniot conditions, rarefaction
branch from the isentropic Riemann invariants), a Newton solve of
f_L(p) + f_R(p) + (u_R - u_L) = 0 for the star pressure, and self-similar
sampling of the wave pattern at x/t.

Test infrastructure: an independent check of the oracle's hydro stage.
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pK, aK, g):
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        s = math.sqrt(A / (p + B))
        return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (B + p))
    r = p / pK  # rarefaction
    f = 2.0 * aK / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * aK) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(WL, WR, g):
    """Return (p*, u*) for primitive states W = (rho, u, p)."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    if 2.0 * (aL + aR) / (g - 1.0) <= uR - uL:
        raise ValueError("vacuum generated")
    p = max(1e-12, 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rL + rR) * (aL + aR))
    for _ in range(200):
        fL, dL = _fK(p, rL, pL, aL, g)
        fR, dR = _fK(p, rR, pR, aR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(1e-14, p - dp)
        if abs(pn - p) <= 1e-15 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, aL, g)
    fR, _ = _fK(p, rR, pR, aR, g)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def star_densities(WL, WR, g):
    p, u = star_state(WL, WR, g)
    out = []
    for (r, _, pK) in (WL, WR):
        if p > pK:
            q = p / pK
            G = (g - 1.0) / (g + 1.0)
            out.append(r * (q + G) / (G * q + 1.0))
        else:
            out.append(r * (p / pK) ** (1.0 / g))
    return p, u, out[0], out[1]


def sample(WL, WR, g, xi):
    """Primitive state (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    ps, us = star_state(WL, WR, g)
    G = (g - 1.0) / (g + 1.0)
    out = np.zeros((len(xi), 3))
    for n, s in enumerate(np.asarray(xi, dtype=float)):
        if s <= us:  # left of the contact
            if ps > pL:
                SL = uL - aL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if s <= SL:
                    out[n] = (rL, uL, pL)
                else:
                    q = ps / pL
                    out[n] = (rL * (q + G) / (G * q + 1.0), us, ps)
            else:
                head = uL - aL
                tail = us - aL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                if s <= head:
                    out[n] = (rL, uL, pL)
                elif s >= tail:
                    out[n] = (rL * (ps / pL) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (aL + 0.5 * (g - 1.0) * uL + s)
                    a = 2.0 / (g + 1.0) * (aL + 0.5 * (g - 1.0) * (uL - s))
                    out[n] = (rL * (a / aL) ** (2.0 / (g - 1.0)), u, pL * (a / aL) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pR:
                SR = uR + aR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if s >= SR:
                    out[n] = (rR, uR, pR)
                else:
                    q = ps / pR
                    out[n] = (rR * (q + G) / (G * q + 1.0), us, ps)
            else:
                head = uR + aR
                tail = us + aR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                if s >= head:
                    out[n] = (rR, uR, pR)
                elif s <= tail:
                    out[n] = (rR * (ps / pR) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-aR + 0.5 * (g - 1.0) * uR + s)
                    a = 2.0 / (g + 1.0) * (aR - 0.5 * (g - 1.0) * (uR - s))
                    out[n] = (rR * (a / aR) ** (2.0 / (g - 1.0)), u, pR * (a / aR) ** (2.0 * g / (g - 1.0)))
    return out
