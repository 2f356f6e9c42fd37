"""Exact Riemann solver for the ideal-gas Euler equations (textbook closed form,
as described for the Riemann problem background in Sec. 4.1.2 of the paper:
three waves, shock or rarefaction on each side, iterative star pressure).

Written independently of the oracle, as a pin: the star pressure solves
f_L(p) + f_R(p) + (u_R - u_L) = 0 with the standard shock (Rankine-Hugoniot)
and rarefaction (isentropic) branches; the solution is sampled at x/t.
"""
from __future__ import annotations

import math


def _f(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star(rl, ul, pl, rr, ur, pr, gamma, tol=1e-15):
    """Star pressure and velocity by bisection + secant polish (robust, slow)."""
    g = lambda p: _f(p, rl, pl, gamma) + _f(p, rr, pr, gamma) + (ur - ul)
    lo, hi = 1e-14, 10.0 * max(pl, pr) + 10.0 * (rl + rr) * (abs(ul) + abs(ur) + 1.0) ** 2
    while g(hi) < 0:
        hi *= 2.0
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            hi = mid
        else:
            lo = mid
        if hi - lo <= tol * hi:
            break
    p = 0.5 * (lo + hi)
    u = 0.5 * (ul + ur) + 0.5 * (_f(p, rr, pr, gamma) - _f(p, rl, pl, gamma))
    return p, u


def sample(rl, ul, pl, rr, ur, pr, gamma, s):
    """(rho, u, p) of the exact solution at x/t = s."""
    ps, us = star(rl, ul, pl, rr, ur, pr, gamma)
    gm1, gp1 = gamma - 1.0, gamma + 1.0
    if s <= us:
        rho, u, p = rl, ul, pl
        c = math.sqrt(gamma * p / rho)
        if ps > p:
            S = u - c * math.sqrt(gp1 / (2 * gamma) * ps / p + gm1 / (2 * gamma))
            if s <= S:
                return rho, u, p
            return rho * (ps / p + gm1 / gp1) / (gm1 / gp1 * ps / p + 1.0), us, ps
        cs = c * (ps / p) ** (gm1 / (2 * gamma))
        if s <= u - c:
            return rho, u, p
        if s >= us - cs:
            return rho * (ps / p) ** (1.0 / gamma), us, ps
        k = 2.0 / gp1 + gm1 / (gp1 * c) * (u - s)
        return rho * k ** (2.0 / gm1), 2.0 / gp1 * (c + gm1 / 2.0 * u + s), p * k ** (2.0 * gamma / gm1)
    rho, u, p = rr, ur, pr
    c = math.sqrt(gamma * p / rho)
    if ps > p:
        S = u + c * math.sqrt(gp1 / (2 * gamma) * ps / p + gm1 / (2 * gamma))
        if s >= S:
            return rho, u, p
        return rho * (ps / p + gm1 / gp1) / (gm1 / gp1 * ps / p + 1.0), us, ps
    cs = c * (ps / p) ** (gm1 / (2 * gamma))
    if s >= u + c:
        return rho, u, p
    if s <= us + cs:
        return rho * (ps / p) ** (1.0 / gamma), us, ps
    k = 2.0 / gp1 - gm1 / (gp1 * c) * (u - s)
    return rho * k ** (2.0 / gm1), 2.0 / gp1 * (-c + gm1 / 2.0 * u + s), p * k ** (2.0 * gamma / gm1)
