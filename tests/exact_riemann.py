"""Exact solution of the 1-D Riemann problem of a gamma-law gas (Toro 1997, ch. 4), test-side only.

The paper compares its Sod run with "the exact Riemann solver in Toro 1997" (§3.2.1).  This is an
independent restatement of that textbook solver, used to pin the oracle: it shares nothing with
oracle/ (different pressure functions, root finder and sampling).  Pinned itself by the closed forms in
tests/test_exact_riemann.py.
"""
import math

from scipy.optimize import brentq


def _fK(p, rho, pK, gamma):
    """Velocity change across the K wave as a function of the star pressure (Toro eqs. 4.6-4.7)."""
    c = math.sqrt(gamma * pK / rho)
    if p > pK:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pK) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(rl, ul, pl, rr, ur, pr, gamma=1.4):
    """(p*, u*) of the exact solution."""
    def f(p):
        return _fK(p, rl, pl, gamma) + _fK(p, rr, pr, gamma) + (ur - ul)

    lo, hi = 1e-300, max(pl, pr)
    if f(lo) >= 0.0:
        raise ValueError("the initial states generate a vacuum")
    while f(hi) < 0.0:
        hi *= 2.0
    ps = brentq(f, lo, hi, xtol=1e-300, rtol=4.0 * 2.0 ** -52, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_fK(ps, rr, pr, gamma) - _fK(ps, rl, pl, gamma))
    return ps, us


def sample(xi, rl, ul, pl, rr, ur, pr, gamma=1.4, star=None):
    """State (rho, u, p) of the exact solution at similarity coordinate xi = x/t."""
    ps, us = star if star is not None else star_state(rl, ul, pl, rr, ur, pr, gamma)
    g = gamma
    gm, gp = g - 1.0, g + 1.0
    if xi <= us:  # left of the contact
        c = math.sqrt(g * pl / rl)
        if ps > pl:  # left shock
            S = ul - c * math.sqrt(gp / (2 * g) * ps / pl + gm / (2 * g))
            if xi <= S:
                return rl, ul, pl
            return rl * (ps / pl + gm / gp) / (gm / gp * ps / pl + 1.0), us, ps
        # left rarefaction
        cs = c * (ps / pl) ** (gm / (2 * g))
        SH, ST = ul - c, us - cs
        if xi <= SH:
            return rl, ul, pl
        if xi >= ST:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        fac = 2.0 / gp + gm / (gp * c) * (ul - xi)
        return rl * fac ** (2.0 / gm), 2.0 / gp * (c + gm / 2.0 * ul + xi), pl * fac ** (2.0 * g / gm)
    c = math.sqrt(g * pr / rr)
    if ps > pr:  # right shock
        S = ur + c * math.sqrt(gp / (2 * g) * ps / pr + gm / (2 * g))
        if xi >= S:
            return rr, ur, pr
        return rr * (ps / pr + gm / gp) / (gm / gp * ps / pr + 1.0), us, ps
    cs = c * (ps / pr) ** (gm / (2 * g))
    SH, ST = ur + c, us + cs
    if xi >= SH:
        return rr, ur, pr
    if xi <= ST:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    fac = 2.0 / gp - gm / (gp * c) * (ur - xi)
    return rr * fac ** (2.0 / gm), 2.0 / gp * (-c + gm / 2.0 * ur + xi), pr * fac ** (2.0 * g / gm)


def cell_averaged_density(x_edges, t, x0, left, right, gamma=1.4, sub=16):
    """Density of the exact solution averaged over cells [x_edges[i], x_edges[i+1]] with sub points each."""
    rl, ul, pl = left
    rr, ur, pr = right
    star = star_state(rl, ul, pl, rr, ur, pr, gamma)
    out = []
    for a, b in zip(x_edges[:-1], x_edges[1:]):
        s = 0.0
        for m in range(sub):
            x = a + (m + 0.5) * (b - a) / sub
            s += sample((x - x0) / t, rl, ul, pl, rr, ur, pr, gamma, star)[0]
        out.append(s / sub)
    return out
