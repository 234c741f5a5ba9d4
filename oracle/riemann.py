"""Exact solution of the 1-D Riemann problem of an ideal gas.

Test infrastructure (oracle side).  Used to pin the oracle on the shock-tube
problem of Sec. 4.2: the initial discontinuity breaks into a left wave
(rarefaction or shock), a contact and a right wave; the star-region pressure
p* is the root of

    f_L(p) + f_R(p) + (v_R - v_L) = 0,

with, for side K of density rho_K, pressure p_K and sound speed c_K,

    f_K(p) = (p - p_K) sqrt(A_K / (p + B_K))            if p > p_K (shock),
    A_K = 2 / ((gamma+1) rho_K),  B_K = p_K (gamma-1)/(gamma+1),
    f_K(p) = 2 c_K/(gamma-1) ((p/p_K)^((gamma-1)/(2 gamma)) - 1)   otherwise,

and v* = (v_L + v_R)/2 + (f_R(p*) - f_L(p*))/2.  The self-similar solution
is then sampled at xi = (x - x0)/t: shock speeds follow from the
Rankine-Hugoniot conditions, rarefaction fans from the isentropic Riemann
invariants.  (Standard gas dynamics, written from the equations above.)
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, gamma):
    c = np.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = pk * (gamma - 1.0) / (gamma + 1.0)
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma):
    """(p*, v*) for left/right primitive states (rho, v, p)."""
    rl, vl, pl = left
    rr, vr, pr = right
    g = lambda p: _f(p, rl, pl, gamma) + _f(p, rr, pr, gamma) + (vr - vl)
    hi = max(pl, pr)
    while g(hi) < 0:
        hi *= 2.0
    ps = brentq(g, 1e-14 * min(pl, pr), hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    vs = 0.5 * (vl + vr) + 0.5 * (_f(ps, rr, pr, gamma) - _f(ps, rl, pl, gamma))
    return ps, vs


def sample(left, right, gamma, xi):
    """Primitive (rho, v, p) arrays at similarity coordinates xi = x/t."""
    rl, vl, pl = left
    rr, vr, pr = right
    ps, vs = star_state(left, right, gamma)
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    gm, gp = gamma - 1.0, gamma + 1.0
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    v = np.empty_like(xi)
    p = np.empty_like(xi)
    for i, s in np.ndenumerate(xi):
        if s <= vs:   # left of the contact
            if ps > pl:   # left shock
                rs = rl * ((ps / pl + gm / gp) / (gm / gp * ps / pl + 1.0))
                S = vl - cl * np.sqrt(gp / (2 * gamma) * ps / pl + gm / (2 * gamma))
                st = (rl, vl, pl) if s <= S else (rs, vs, ps)
            else:         # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                cs = cl * (ps / pl) ** (gm / (2 * gamma))
                head, tail = vl - cl, vs - cs
                if s <= head:
                    st = (rl, vl, pl)
                elif s >= tail:
                    st = (rs, vs, ps)
                else:
                    c = 2.0 / gp * (cl + gm / 2.0 * (vl - s))
                    vv = 2.0 / gp * (cl + gm / 2.0 * vl + s)
                    rr_ = rl * (c / cl) ** (2.0 / gm)
                    st = (rr_, vv, pl * (c / cl) ** (2.0 * gamma / gm))
        else:         # right of the contact
            if ps > pr:   # right shock
                rs = rr * ((ps / pr + gm / gp) / (gm / gp * ps / pr + 1.0))
                S = vr + cr * np.sqrt(gp / (2 * gamma) * ps / pr + gm / (2 * gamma))
                st = (rr, vr, pr) if s >= S else (rs, vs, ps)
            else:         # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                cs = cr * (ps / pr) ** (gm / (2 * gamma))
                head, tail = vr + cr, vs + cs
                if s >= head:
                    st = (rr, vr, pr)
                elif s <= tail:
                    st = (rs, vs, ps)
                else:
                    c = 2.0 / gp * (cr - gm / 2.0 * (vr - s))
                    vv = 2.0 / gp * (-cr + gm / 2.0 * vr + s)
                    rr_ = rr * (c / cr) ** (2.0 / gm)
                    st = (rr_, vv, pr * (c / cr) ** (2.0 * gamma / gm))
        rho[i], v[i], p[i] = st
    return rho, v, p


def wave_positions(left, right, gamma):
    """Speeds of the contact and of the shock (right-moving shock assumed,
    as in the Sod problem) and the rarefaction head/tail speeds."""
    rl, vl, pl = left
    rr, vr, pr = right
    ps, vs = star_state(left, right, gamma)
    gm, gp = gamma - 1.0, gamma + 1.0
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    S = vr + cr * np.sqrt(gp / (2 * gamma) * ps / pr + gm / (2 * gamma))
    cs = cl * (ps / pl) ** (gm / (2 * gamma))
    return {"contact": vs, "shock": S, "rare_head": vl - cl, "rare_tail": vs - cs, "p_star": ps}
