"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations
(Newton iteration on the pressure function, the method of Toro's book, which
the paper uses for its shock-tube reference solutions, Sec. 3.2)."""
import math

import numpy as np


def _fk(p, rk, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (p + B)) * (1.0 - (p - pk) / (2.0 * (B + p)))
    else:
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rk * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, g=1.4):
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = 0.5 * (pl + pr)
    for _ in range(200):
        f1, d1 = _fk(p, rl, pl, cl, g)
        f2, d2 = _fk(p, rr, pr, cr, g)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p = max(p - dp, 1e-14)
        if abs(dp) < 1e-15 * p:
            break
    u = 0.5 * (ul + ur) + 0.5 * (_fk(p, rr, pr, cr, g)[0] - _fk(p, rl, pl, cl, g)[0])
    if p > pl:
        rsl = rl * ((p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1))
    else:
        rsl = rl * (p / pl) ** (1.0 / g)
    if p > pr:
        rsr = rr * ((p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1))
    else:
        rsr = rr * (p / pr) ** (1.0 / g)
    return p, u, rsl, rsr


def sample(x, t, x0, left, right, g=1.4):
    """Primitive (rho, u, p) at positions x, time t, for a left rarefaction /
    right shock configuration such as Sod's."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us, rsl, rsr = star_state(rl, ul, pl, rr, ur, pr, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    csl = math.sqrt(g * ps / rsl)
    S = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
    out = np.empty((len(x), 3))
    for k, xx in enumerate(x):
        s = (xx - x0) / t
        if s < ul - cl:
            out[k] = (rl, ul, pl)
        elif s < us - csl:
            r = rl * (2 / (g + 1) + (g - 1) / ((g + 1) * cl) * (ul - s)) ** (2 / (g - 1))
            u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
            p = pl * (2 / (g + 1) + (g - 1) / ((g + 1) * cl) * (ul - s)) ** (2 * g / (g - 1))
            out[k] = (r, u, p)
        elif s < us:
            out[k] = (rsl, us, ps)
        elif s < S:
            out[k] = (rsr, us, ps)
        else:
            out[k] = (rr, ur, pr)
    return out
