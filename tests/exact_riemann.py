"""Exact solution of the 1D Riemann problem for an ideal gas.

Written independently of the oracle to pin it: the pressure function of
Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics" (Ch. 4,
Eqs. 4.5-4.8), solved for p* by Newton iteration, and the self-similar
sampling of the wave fan at xi = (x - x0) / t (Sec. 4.5).
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho_k, p_k, c_k, g):
    """Pressure function f_K(p) and its derivative for one side."""
    if p > p_k:  # shock
        a = 2.0 / ((g + 1.0) * rho_k)
        b = (g - 1.0) / (g + 1.0) * p_k
        q = math.sqrt(a / (p + b))
        return (p - p_k) * q, q * (1.0 - 0.5 * (p - p_k) / (b + p))
    # rarefaction
    r = p / p_k
    f = 2.0 * c_k / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho_k * c_k) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4, tol=1e-15):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum generated")
    p = max(tol, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        f = fl + fr + (ur - ul)
        p_new = p - f / (dfl + dfr)
        if p_new < tol:
            p_new = tol
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, left, right, g=1.4):
    """Primitive (rho, u, p) of the exact solution at xi = x/t (scalar)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    gm = (g - 1.0) / (g + 1.0)
    if xi <= us:  # left of the contact
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            if xi <= sl:
                return rl, ul, pl
            rho = rl * ((ps / pl + gm) / (gm * ps / pl + 1.0))
            return rho, us, ps
        # left rarefaction
        cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        head, tail = ul - cl, us - cs
        if xi <= head:
            return rl, ul, pl
        if xi >= tail:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi))
        u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + xi)
        rho = rl * (c / cl) ** (2.0 / (g - 1.0))
        p = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        return rho, u, p
    # right of the contact
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        if xi >= sr:
            return rr, ur, pr
        rho = rr * ((ps / pr + gm) / (gm * ps / pr + 1.0))
        return rho, us, ps
    cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    head, tail = ur + cr, us + cs
    if xi >= head:
        return rr, ur, pr
    if xi <= tail:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - xi))
    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + xi)
    rho = rr * (c / cr) ** (2.0 / (g - 1.0))
    p = pr * (c / cr) ** (2.0 * g / (g - 1.0))
    return rho, u, p


def cell_average_density(n, t, left, right, x0=0.5, g=1.4, sub=64):
    """Exact density averaged over each of n cells of [0, 1] (midpoint rule
    with `sub` points per cell)."""
    dx = 1.0 / n
    out = np.empty(n)
    for i in range(n):
        xs = i * dx + (np.arange(sub) + 0.5) * dx / sub
        out[i] = np.mean([sample((x - x0) / t, left, right, g)[0] for x in xs])
    return out
