"""Exact solution of the 1D Riemann problem for an ideal gas (TEST INFRASTRUCTURE ONLY).

Written from the definition of the Riemann problem of the Euler equations:
the star pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is
the velocity jump across a shock (p > p_K, Rankine-Hugoniot conditions) or an
isentropic rarefaction (p <= p_K, Riemann invariants); u* follows from the
same functions and the solution is self-similar in x/t.

It is the xi = 1 reference of the shock-tube check (the RSST at xi = 1 is the
conservative Euler system, Sec. 3.2).  Its star state is pinned against the
values the textbook literature prints for the Sod problem
(tests/golden/sod_star_state.json).
"""
from __future__ import annotations

import math


def _f(p, rho, pk, gamma):
    """Velocity jump across the wave on one side at star pressure p: a shock
    (Rankine-Hugoniot) for p > pk, an isentropic rarefaction otherwise."""
    a = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * a / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(rl, ul, pl, rr, ur, pr, gamma):
    """Return (p*, u*) by bisection on the monotone pressure function."""
    g = lambda p: _f(p, rl, pl, gamma) + _f(p, rr, pr, gamma) + (ur - ul)
    lo, hi = 1e-14, max(pl, pr)
    while g(hi) < 0.0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    p = 0.5 * (lo + hi)
    u = 0.5 * (ul + ur) + 0.5 * (_f(p, rr, pr, gamma) - _f(p, rl, pl, gamma))
    return p, u


def star_densities(rl, pl, rr, pr, p, gamma):
    """Densities either side of the contact: shock adiabat or isentrope."""
    def rho_star(rk, pk):
        if p > pk:
            q = (gamma - 1.0) / (gamma + 1.0)
            return rk * (p / pk + q) / (q * p / pk + 1.0)
        return rk * (p / pk) ** (1.0 / gamma)
    return rho_star(rl, pl), rho_star(rr, pr)


def sample(s, rl, ul, pl, rr, ur, pr, gamma):
    """(rho, u, p) at similarity coordinate s = (x - x0)/t."""
    p, u = star_state(rl, ul, pl, rr, ur, pr, gamma)
    rls, rrs = star_densities(rl, pl, rr, pr, p, gamma)
    if s <= u:  # left of the contact
        a = math.sqrt(gamma * pl / rl)
        if p > pl:
            shock = ul - a * math.sqrt((gamma + 1) / (2 * gamma) * p / pl + (gamma - 1) / (2 * gamma))
            return (rl, ul, pl) if s < shock else (rls, u, p)
        head = ul - a
        tail = u - a * (p / pl) ** ((gamma - 1) / (2 * gamma))
        if s < head:
            return rl, ul, pl
        if s > tail:
            return rls, u, p
        uu = 2.0 / (gamma + 1) * (a + (gamma - 1) / 2 * ul + s)
        c = 2.0 / (gamma + 1) * (a + (gamma - 1) / 2 * (ul - s))
        rho = rl * (c / a) ** (2.0 / (gamma - 1))
        return rho, uu, pl * (c / a) ** (2 * gamma / (gamma - 1))
    a = math.sqrt(gamma * pr / rr)
    if p > pr:
        shock = ur + a * math.sqrt((gamma + 1) / (2 * gamma) * p / pr + (gamma - 1) / (2 * gamma))
        return (rr, ur, pr) if s > shock else (rrs, u, p)
    head = ur + a
    tail = u + a * (p / pr) ** ((gamma - 1) / (2 * gamma))
    if s > head:
        return rr, ur, pr
    if s < tail:
        return rrs, u, p
    uu = 2.0 / (gamma + 1) * (-a + (gamma - 1) / 2 * ur + s)
    c = 2.0 / (gamma + 1) * (a - (gamma - 1) / 2 * (ur - s))
    rho = rr * (c / a) ** (2.0 / (gamma - 1))
    return rho, uu, pr * (c / a) ** (2 * gamma / (gamma - 1))
