"""Exact solution of the 1D Euler Riemann problem for an ideal gas (test helper).

Textbook method (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4):
the star-region pressure p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is
the shock (Rankine-Hugoniot) or rarefaction (isentropic) relation of side K; the solution
is then sampled along rays x/t.  Used to pin the oracle's Sod shock tube.
"""

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, c, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(left, right, g):
    """(p*, u*) for left/right states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    fn = lambda p: _f(p, rl, pl, cl, g) + _f(p, rr, pr, cr, g) + (ur - ul)
    p = brentq(fn, 1e-12 * min(pl, pr), 10.0 * max(pl, pr), xtol=1e-15, rtol=1e-15)
    u = 0.5 * (ul + ur) + 0.5 * (_f(p, rr, pr, cr, g) - _f(p, rl, pl, cl, g))
    return p, u


def sample(left, right, g, xi):
    """(rho, u, p) at similarity coordinates xi = x/t.  Handles a left rarefaction and a
    right shock (the Sod structure), which is all the tests use."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    assert ps < pl and ps > pr, "only left-rarefaction / right-shock problems are sampled"
    rho_sl = rl * (ps / pl) ** (1.0 / g)
    gm = (g - 1.0) / (g + 1.0)
    rho_sr = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
    s_shock = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
    s_head = ul - cl
    s_tail = us - cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
    xi = np.asarray(xi, dtype=float)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, x in np.ndenumerate(xi):
        if x < s_head:
            rho[k], u[k], p[k] = rl, ul, pl
        elif x < s_tail:
            fac = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * cl) * (ul - x)
            rho[k] = rl * fac ** (2.0 / (g - 1.0))
            u[k] = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + x)
            p[k] = pl * fac ** (2.0 * g / (g - 1.0))
        elif x < us:
            rho[k], u[k], p[k] = rho_sl, us, ps
        elif x < s_shock:
            rho[k], u[k], p[k] = rho_sr, us, ps
        else:
            rho[k], u[k], p[k] = rr, ur, pr
    return rho, u, p, dict(p_star=ps, u_star=us, s_shock=s_shock, s_head=s_head, s_tail=s_tail,
                           rho_star_left=rho_sl, rho_star_right=rho_sr)
