"""Pins of the oracle's shock detector and DWBAP limiter (Sec. III.C): smooth
data are not flagged and keep their coefficients; the limited scheme runs the
Sod problem (Eq. (44)) to t = 0.2 with positive states, and its distance to the
exact Riemann solution (Rankine-Hugoniot and isentropic relations, solved by
Newton iteration on the star pressure) shrinks under mesh refinement."""
import math

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I

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


def test_exact_riemann_solver_star_state():
    # Sod: star pressure 0.30313 and velocity 0.92745 (textbook values of the problem)
    x = np.array([0.5 + 0.92745 * 0.2 - 1e-4])
    r, u, p = exact_riemann(x, 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p[0] - 0.30313) < 1e-4 and abs(u[0] - 0.92745) < 1e-4


def test_smooth_data_not_limited(oracle_mod):
    c = I.advection_case(16)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1)
    coef, _, _, _ = om.cls_solve(c.w0)
    lim, flag = om.limit(c.w0, coef)
    assert np.all(flag == 0) and np.array_equal(lim, coef)


def _sod_l1(oracle_mod, nx, ny):
    c = I.sod_case(nx, ny)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1)
    w = c.w0.copy()
    t = 0.0
    while t < 0.2 - 1e-14:
        dt = min(om.cfl_dt(w), 0.2 - t)
        info = om.step(w, dt)
        assert info.status == 0
        t += dt
    cg = om.cell_geometry()
    ex = exact_riemann(cg["cx"], 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    p = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
    assert np.all(w[0] > 0) and np.all(p > 0)
    area = cg["area"]
    return np.sum(area * np.abs(w[0] - ex[0])) / area.sum()


def test_limited_sod_converges_to_exact_riemann(oracle_mod):
    e1 = _sod_l1(oracle_mod, 40, 3)
    e2 = _sod_l1(oracle_mod, 80, 6)
    assert e2 < e1 / 1.4 and e2 < 0.01, (e1, e2)


def test_limiter_flags_only_near_the_jump(oracle_mod):
    c = I.sod_case(100, 4)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1)
    coef, _, _, _ = om.cls_solve(c.w0)
    lim, flag = om.limit(c.w0, coef)
    cx = om.cell_geometry()["cx"]
    assert flag.sum() > 0
    assert np.all(np.abs(cx[flag > 0] - 0.5) < 0.05)
    assert np.array_equal(lim[:, :, flag == 0], coef[:, :, flag == 0])
