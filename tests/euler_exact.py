"""Exact Riemann solution of the 1D Euler equations of an ideal gas (Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4: pressure function, Newton iteration for p*, and
sampling of the self-similar solution).  Used as the eps -> 0 limit of the kinetic scheme; for
d_v = 2 the limit gas has gamma = (d_v + 2) / d_v = 2."""
import math

import numpy as np


def _fK(p, rho, pK, a, g):
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        s = math.sqrt(A / (p + B))
        return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (B + p))
    r = p / pK
    f = 2.0 * a / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    d = 1.0 / (rho * a) * r ** (-(g + 1.0) / (2.0 * g))
    return f, d


def star_state(L, R, g):
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _fK(p, rl, pl, al, g)
        fr, dr = _fK(p, rr, pr, ar, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        pn = max(pn, 1e-12)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, al, g)
    fr, _ = _fK(p, rr, pr, ar, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(L, R, g, xi):
    """(rho, u, p) at xi = (x - x0) / t."""
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(L, R, g)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:
            if ps > pl:
                sl = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    out[:, n] = (rl, ul, pl)
                else:
                    rs = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                    out[:, n] = (rs, us, ps)
            else:
                ash = al * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - al:
                    out[:, n] = (rl, ul, pl)
                elif s >= us - ash:
                    out[:, n] = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
                    out[:, n] = (rl * c ** (2 / (g - 1)),
                                 2 / (g + 1) * (al + (g - 1) / 2 * ul + s),
                                 pl * c ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                sr = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    out[:, n] = (rr, ur, pr)
                else:
                    rs = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                    out[:, n] = (rs, us, ps)
            else:
                ash = ar * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + ar:
                    out[:, n] = (rr, ur, pr)
                elif s <= us + ash:
                    out[:, n] = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
                    out[:, n] = (rr * c ** (2 / (g - 1)),
                                 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s),
                                 pr * c ** (2 * g / (g - 1)))
    return out
