"""Exact solution of the 1-D Riemann problem of the Euler equations (textbook
construction: the star pressure from the shock and rarefaction curves by Newton
iteration, then sampling of the self-similar solution).  Test helper: an
independent reference for the shock-tube runs of Sec. IV (Sod, Eq. (44))."""
import math

import numpy as np

GAMMA = 1.4


def exact_riemann(x, t, left, right, x0=0.5, g=GAMMA):
    """Exact solution (rho, u, p) of the 1-D Riemann problem (textbook: star
    pressure from the shock / rarefaction curves, then sampling)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def f(p, rk, pk, ck):
        if p > pk:
            A, B = 2 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
            q = math.sqrt(A / (p + B))
            return (p - pk) * q, q * (1 - (p - pk) / (2 * (B + p)))
        e = (g - 1) / (2 * g)
        return 2 * ck / (g - 1) * ((p / pk) ** e - 1), (p / pk) ** (-(g + 1) / (2 * g)) / (rk * ck)

    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = f(p, rl, pl, cl)
        fr, dr = f(p, rr, pr, cr)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    us = 0.5 * (ul + ur) + 0.5 * (f(p, rr, pr, cr)[0] - f(p, rl, pl, cl)[0])
    out = np.zeros((3, x.size))
    for n, xi in enumerate(x):
        s = (xi - x0) / t if t > 0 else (-1e300 if xi < x0 else 1e300)
        if s < us:   # left of the contact
            if p > pl:
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                r = rl * ((p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1))
                out[:, n] = (rl, ul, pl) if s < sl else (r, us, p)
            else:
                csl = cl * (p / pl) ** ((g - 1) / (2 * g))
                if s < ul - cl:
                    out[:, n] = (rl, ul, pl)
                elif s > us - csl:
                    out[:, n] = (rl * (p / pl) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    r = rl * (c / cl) ** (2 / (g - 1))
                    out[:, n] = (r, u, r * c * c / g)
        else:        # right of the contact
            if p > pr:
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
                r = rr * ((p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1))
                out[:, n] = (rr, ur, pr) if s > sr else (r, us, p)
            else:
                csr = cr * (p / pr) ** ((g - 1) / (2 * g))
                if s > ur + cr:
                    out[:, n] = (rr, ur, pr)
                elif s < us + csr:
                    out[:, n] = (rr * (p / pr) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    r = rr * (c / cr) ** (2 / (g - 1))
                    out[:, n] = (r, u, r * c * c / g)
    return out
