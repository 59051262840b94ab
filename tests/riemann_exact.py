"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas with constant ratio of specific heats gamma.

An independent check (pin) of the oracle's shock-tube behaviour, written
from the textbook mathematics: the star-region pressure p* is the root of
f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the Rankine-Hugoniot
velocity jump across a shock (p > p_K) or the isentropic Riemann-invariant
jump across a rarefaction (p <= p_K); the solution is then sampled on the
self-similar variable xi = x / t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * a / (gamma - 1.0) * ((p / pk) ** e - 1.0)
    df = 1.0 / (rho * a) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    """(p*, u*) for left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dfl = _f_and_df(p, rl, pl, gamma)
        fr, dfr = _f_and_df(p, rr, pr, gamma)
        g = fl + fr + (ur - ul)
        pn = max(p - g / (dfl + dfr), 1e-12 * p)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, gamma)
    fr, _ = _f_and_df(p, rr, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, gamma, xi):
    """(rho, u, p) arrays at xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - al * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                if s <= sl:
                    rho[k], u[k], p[k] = rl, ul, pl
                else:
                    rho[k] = rl * ((ps / pl) + g1) / (g1 * (ps / pl) + 1.0)
                    u[k], p[k] = us, ps
            else:  # left rarefaction
                shl = ul - al
                asl = al * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                stl = us - asl
                if s <= shl:
                    rho[k], u[k], p[k] = rl, ul, pl
                elif s >= stl:
                    rho[k] = rl * (ps / pl) ** (1.0 / gamma)
                    u[k], p[k] = us, ps
                else:
                    c = 2.0 / (gamma + 1) + g1 / al * (ul - s)
                    rho[k] = rl * c ** (2.0 / (gamma - 1))
                    u[k] = 2.0 / (gamma + 1) * (al + (gamma - 1) / 2 * ul + s)
                    p[k] = pl * c ** (2.0 * gamma / (gamma - 1))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + ar * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                if s >= sr:
                    rho[k], u[k], p[k] = rr, ur, pr
                else:
                    rho[k] = rr * ((ps / pr) + g1) / (g1 * (ps / pr) + 1.0)
                    u[k], p[k] = us, ps
            else:  # right rarefaction
                shr = ur + ar
                asr = ar * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                str_ = us + asr
                if s >= shr:
                    rho[k], u[k], p[k] = rr, ur, pr
                elif s <= str_:
                    rho[k] = rr * (ps / pr) ** (1.0 / gamma)
                    u[k], p[k] = us, ps
                else:
                    c = 2.0 / (gamma + 1) - g1 / ar * (ur - s)
                    rho[k] = rr * c ** (2.0 / (gamma - 1))
                    u[k] = 2.0 / (gamma + 1) * (-ar + (gamma - 1) / 2 * ur + s)
                    p[k] = pr * c ** (2.0 * gamma / (gamma - 1))
    return rho, u, p
