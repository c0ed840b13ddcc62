"""Exact solution of the 1D Riemann problem for the Euler equations of an ideal gas.

Written from the mathematics of the problem as presented in E. F. Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", Ch. 4 (pressure function, Newton iteration for the star
pressure, and sampling of the self-similar solution).  Used only by the tests, as an
independent pin of the oracle on shock problems.
"""
import numpy as np


def _pressure_fn(p, rho, pk, ck, g):
    if p > pk:                                             # shock branch
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:                                                  # rarefaction branch
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * ck)
    return f, df


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _pressure_fn(p, rl, pl, cl, g)
        fr, dfr = _pressure_fn(p, rr, pr, cr, g)
        pn = max(1e-12, p - (fl + fr + ur - ul) / (dfl + dfr))
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _pressure_fn(p, rl, pl, cl, g)
    fr, _ = _pressure_fn(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, g=1.4):
    """Density, velocity and pressure at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    out = np.zeros((3, len(xi)))
    gm = (g - 1.0) / (g + 1.0)
    for k, s in enumerate(xi):
        if s <= us:                                        # left of the contact
            if ps > pl:
                sh = ul - cl * np.sqrt((g + 1.0) / (2 * g) * ps / pl + (g - 1.0) / (2 * g))
                val = (rl, ul, pl) if s <= sh else (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:
                csl = cl * (ps / pl) ** ((g - 1.0) / (2 * g))
                if s <= ul - cl:
                    val = (rl, ul, pl)
                elif s >= us - csl:
                    val = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2 * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2 * (ul - s))
                    val = (rl * (c / cl) ** (2.0 / (g - 1.0)), u, pl * (c / cl) ** (2 * g / (g - 1.0)))
        else:                                              # right of the contact
            if ps > pr:
                sh = ur + cr * np.sqrt((g + 1.0) / (2 * g) * ps / pr + (g - 1.0) / (2 * g))
                val = (rr, ur, pr) if s >= sh else (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:
                csr = cr * (ps / pr) ** ((g - 1.0) / (2 * g))
                if s >= ur + cr:
                    val = (rr, ur, pr)
                elif s <= us + csr:
                    val = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2 * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2 * (ur - s))
                    val = (rr * (c / cr) ** (2.0 / (g - 1.0)), u, pr * (c / cr) ** (2 * g / (g - 1.0)))
        out[:, k] = val
    return out
